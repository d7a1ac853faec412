// k_find.cu — ZS decode + 3x3 peak finder + 5x5 cluster moments + stable
// compaction (steps 1-4 of the library's definition; the paper's section
// "Hardware and data flow" places this first step of the TPC reconstruction on
// the EPN GPUs, after FPGA zero suppression).
//
// A window is (sector, row, 256-bin fragment) with 3-bin halos from both
// neighbouring pages.  k_find_classify sorts the windows by their page
// headers: a light window (at most 256 digits and runs with its halos) goes to
// one warp of k_find_light, the others to the persistent block finder
// k_find_clusters; the two run side by side on two streams.
// Block finder: one CTA iteration per window.  The page, both halo byte ranges
// and the own header travel in one round trip (the neighbours' headers were
// copied during the previous window); everything after that reads shared
// memory.  Digits are decoded (entries, runs, digits in balanced block-wide
// phases) into a zero-padded plane (two empty pads on each side of the row)
// kept empty between windows: a listed window resets only the cells its digits
// wrote, a dense one clears the plane with 16-byte stores, so every pixel
// lookup is a single shared load.  The peak test runs one thread per listed
// digit (dense windows: equal shares of the occupied pixels); own peaks are
// ranked in canonical (t, pad) order by popcount prefixes over the peak
// bitmap, and one thread per peak builds its cluster from the 5x5
// neighbourhood held in registers.  Each window reserves a span of a scratch
// buffer with one atomic; a scan of the window counts and a compaction place
// the records canonically.  The allocation-free entry point instead gives each
// window its offset by a decoupled look-back over the windows.
#include <algorithm>
#include <mutex>

#include "find_common.cuh"

namespace tpc {

constexpr int kFindThreads = 384;   // default block size (the allocation-free entry point's)

constexpr int kStage = 256;                  // clusters staged in shared memory before the look-back
// The own page is staged in [st_rec | st_xyz | plist | ppre], contiguous and
// unused until the decode is over: 2 * kStage * 16 + kStage * 2 bytes plus
// the rank prefix (own_stage_bytes).
constexpr int kHaloStage = 2048;             // bytes per neighbouring page's halo ranges
constexpr int kHaloRunOff = 16, kHaloAdcOff = 800;
constexpr int kList = 4096;                  // digits listed by the decoder (beyond: bitmap walk)
constexpr int kDenseU = 7;                   // dense-plane chunks a thread has in flight
constexpr int kMaxRuns = 2048;               // runs of a window decoded run-parallel (beyond: per entry)
constexpr int kRunMapWords = kList / 32;     // run-start bitmap over the listed digits
// Windows with more than kList digits (a dense row) are decoded the same
// balanced way, the list area then holding, instead of one plane index per
// digit, one per run (run_L), the run-start bitmap over up to kMaxDig digits
// and the run starts before each bitmap word; they skip the digit list.
constexpr int kMaxDig = 16384;
constexpr int kBigWords = kMaxDig / 32;
static_assert(kMaxRuns * 2 + kBigWords * 4 + kBigWords * 2 <= kList * 2, "the big-window maps fit the list area");

struct FindSmem {
  uint16_t* plane;     // [kWinT][ps], pixel (tt, p) at tt * ps + p + kPad; zero where no digit
  uint32_t* occ;       // [kWinT][nw] occupancy bitmap
  uint32_t* pk;        // [kWinT][nw] peak bitmap
  uint32_t* dbm;       // [kRunMapWords] bit d set: listed digit d starts a run (follows pk)
  uint8_t* run_t;      // [kMaxRuns] time bin (within its page) of each run of the window
  uint16_t* list;      // [kList] plane index of every decoded digit
  uint16_t* plist;     // [kStage] plane index of the first own peaks in canonical order
  uint16_t* ppre;      // own-peak rank prefix over the words of rows 3..258
  uint4* st_rec;       // [kStage] staged cluster records (first: the staged page)
  int4* st_xyz;        // [kStage] staged (X, Y, Z, t_peak)
  uint8_t* halo;       // [2][kHaloStage] halo ranges of the previous / next page
  uint4* hdr;          // [4] headers of the previous (0,1) and next (2,3) page
  unsigned long long* offs;  // [4] page offsets of windows w-1 .. w+2
  unsigned long long* scan;  // [34]
  int32_t* misc;       // [16]
  PageHdr* ph;         // [3] parsed headers: own, previous, next page
};

// R(a, b) = floor((2a + b) / (2b)), b > 0
__device__ __forceinline__ long long round_half_up(long long a, long long b) {
  long long n = 2 * a + b, d = 2 * b;
  long long q = n / d;
  if ((n % d) != 0 && (n < 0)) q -= 1;
  return q;
}
// Entries of one page to decode: entries (t_in | n_runs << 8), the runs they
// own (pad_start | len << 8) and their ADC words; digit k of the segment is
// field (dfirst + k) % 3 of word (dfirst + k) / 3.  Digit k is listed at
// list[lbase + k] if that is below kList.  Pointers may be shared or global.
struct Seg {
  const uint16_t* ent; int ne;
  const uint16_t* run; int nrun;
  const uint32_t* adc; int dfirst; int ndig;
  int tt_base, t_base_abs, lbase;
  bool strict;                    // the window's own page: ordering and exact counts
};

// Occupancy bits of pads [ps, ps + len) of plane row tt.
__device__ __forceinline__ void set_occ(const FindSmem& S, int nw, int tt, int ps, int len) {
  int p = ps;
  const int pe = ps + len;
  while (p < pe) {
    const int wi = p >> 5, b0 = p & 31;
    const int n = min(32 - b0, pe - p);
    const uint32_t m = (n == 32) ? 0xffffffffu : (((1u << n) - 1u) << b0);
    atomicOr(&S.occ[tt * nw + wi], m);
    p += n;
  }
}

__device__ __forceinline__ void put_run(const Seg& g, const FindSmem& S, int ps_stride, int nw, int tt, int ps,
                                        int len, int di) {
  uint16_t* prow = S.plane + tt * ps_stride + kPad + ps;
  const int d0 = g.dfirst + di;
  int wd = d0 / 3, sh = 10 * (d0 - 3 * (d0 / 3));
  uint32_t word = g.adc[wd];
  const int li0 = g.lbase + di;
  const uint16_t L0 = (uint16_t)(tt * ps_stride + kPad + ps);
  const bool list_all = li0 + len <= kList;
  for (int k = 0; k < len; k++) {
    prow[k] = (uint16_t)((word >> sh) & 1023u);
    if (list_all) S.list[li0 + k] = (uint16_t)(L0 + k);
    else if (li0 + k < kList) S.list[li0 + k] = (uint16_t)(L0 + k);
    sh += 10;
    if (sh == 30 && k + 1 < len) { sh = 0; word = g.adc[++wd]; }
  }
  set_occ(S, nw, tt, ps, len);
}

__device__ __forceinline__ bool decode_seg_warp(const Seg& g, int np, int ps_stride, int nw, int T, const FindSmem& S);

// Block-wide decode of the own page into plane rows tt = t_in + tt_base, one
// thread per time-bin entry (a page has at most 256): a block scan of the run
// counts gives each entry its first run, a second of the digit counts its first
// digit.  When the digits are listed, each entry thread then only writes the
// plane index of its digits into the list, and the block writes the ADC values
// digit-parallel (an entry can hold ten times the mean number of digits);
// otherwise each entry thread writes its digits.  The halo segments (hprev,
// hnext; may be null) are decoded meanwhile by the last two warps.  All reads
// are bounds-checked against the segment's counts and all writes against the
// plane.  Returns true (block-uniform) if valid (own_ok and every check passed).
__device__ __forceinline__ bool decode_seg(const Seg& g, bool own_ok, int np, int ps_stride, int nw, int T, const FindSmem& S,
                           const Seg* hprev, const Seg* hnext) {
  const int tid = threadIdx.x;
  const int ne = own_ok ? g.ne : 0;
  bool bad = !own_ok || ne < 0 || ne > kFrag || ne > (int)blockDim.x;
  const bool mine = !bad && tid < ne;
  int t_in = 0, nr = 0, tt = 0;
  if (mine) {
    const uint32_t v = g.ent[tid];
    t_in = v & 0xff;
    nr = v >> 8;
    tt = t_in + g.tt_base;
    if (nr < 1 || tt < 0 || tt >= kWinT || g.t_base_abs + t_in >= T) { bad = true; nr = 0; }
    if (g.strict && tid > 0 && (int)(g.ent[tid - 1] & 0xff) >= t_in) bad = true;
  }
  uint32_t tot;
  const int r0 = (int)block_excl_scan32((uint32_t)nr, reinterpret_cast<uint32_t*>(S.scan), &tot);
  const int nrun = (int)tot;
  if (own_ok && (nrun > g.nrun || (g.strict && nrun != g.nrun))) bad = true;
  // digits of this entry's runs, with the run checks
  int nd = 0;
  if (mine && r0 + nr <= g.nrun) {
    int last_end = -1;
    for (int k = 0; k < nr; k++) {
      const uint32_t rv = g.run[r0 + k];
      const int ps = rv & 0xff, len = rv >> 8;
      if (len < 1 || ps + len > np) { bad = true; nd = 0; break; }
      if (g.strict && ps < last_end) bad = true;
      last_end = ps + len;
      nd += len;
    }
  } else if (mine) {
    bad = true;
  }
  const long long d0 = (long long)block_excl_scan32((uint32_t)nd, reinterpret_cast<uint32_t*>(S.scan) + 20, &tot);
  if (own_ok && ((long long)tot > g.ndig || (g.strict && (long long)tot != g.ndig))) bad = true;
  const bool list_fill = g.lbase == 0 && g.dfirst == 0 && g.ndig <= kList;
  if (mine && nd > 0 && d0 + nd <= g.ndig) {
    int di = (int)d0;
    for (int k = 0; k < nr; k++) {
      const uint32_t rv = g.run[r0 + k];
      const int ps = rv & 0xff, len = rv >> 8;
      if (list_fill) {
        const uint16_t L0 = (uint16_t)(tt * ps_stride + kPad + ps);
        for (int q = 0; q < len; q++) S.list[di + q] = (uint16_t)(L0 + q);
        set_occ(S, nw, tt, ps, len);
      } else {
        put_run(g, S, ps_stride, nw, tt, ps, len, di);
      }
      di += len;
    }
  }
  const int wid = tid >> 5, nwarp = (int)(blockDim.x >> 5);
  if (hprev && wid == nwarp - 2) decode_seg_warp(*hprev, np, ps_stride, nw, T, S);
  if (hnext && wid == nwarp - 1) decode_seg_warp(*hnext, np, ps_stride, nw, T, S);
  const bool valid = !__syncthreads_or(bad);
  if (valid && list_fill) {
    // every own digit d has its plane index in list[d]: write the ADC values
    const int nplane = kWinT * ps_stride;
    for (uint32_t d = tid; d < (uint32_t)g.ndig; d += blockDim.x) {
      const int L = S.list[d];
      const uint32_t word = g.adc[d / 3u];
      if (L < nplane) S.plane[L] = (uint16_t)((word >> (10u * (d % 3u))) & 1023u);
    }
  }
  return valid;
}

// Warp-level decode of a small segment (the 3-bin halos): the same checks, no
// block barrier.  A violated bound stops it; the page's own window reports it.
__device__ __forceinline__ bool decode_seg_warp(const Seg& g, int np, int ps_stride, int nw, int T, const FindSmem& S) {
  const int lane = threadIdx.x & 31;
  bool bad = g.ne < 0 || g.ne > kFrag;
  int run0 = 0, dig0 = 0;   // runs / digits consumed by earlier entries
  for (int e = 0; e < g.ne && !bad; e++) {
    const uint32_t v = g.ent[e];
    const int t_in = v & 0xff, nr = v >> 8;
    const int tt = t_in + g.tt_base;
    if (nr < 1 || tt < 0 || tt >= kWinT || g.t_base_abs + t_in >= T || run0 + nr > g.nrun) { bad = true; break; }
    for (int jb = 0; jb < nr; jb += 32) {
      const int j = jb + lane;
      int ps = 0, len = 0;
      if (j < nr) {
        const uint32_t rv = g.run[run0 + j];
        ps = rv & 0xff;
        len = rv >> 8;
        if (len < 1 || ps + len > np) { len = 0; bad = true; }
      }
      int incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
      }
      const int di = dig0 + incl - len;
      if (len && di + len > g.ndig) { len = 0; bad = true; }
      if (len) put_run(g, S, ps_stride, nw, tt, ps, len, di);
      dig0 += __shfl_sync(0xffffffffu, incl, 31);
      bad = __any_sync(0xffffffffu, bad);
    }
    run0 += nr;
  }
  return !bad;
}

// Balanced decode of a whole window: the previous page's last 3 bins, the own
// page and the next page's first 3 bins as one sequence of entries, runs and
// digits (segments 0, 1, 2; listed in that order).  Three parallel phases, so
// that no thread holds a whole time bin (an entry can hold ten times the mean
// number of digits per thread):
//   entries (two per thread at most): checks, run counts -> block scan -> run
//     offsets; each entry tags its runs with its time bin;
//   runs (a contiguous block per thread): checks, digit counts -> block scan ->
//     digit offsets; each run lists the plane index of its first digit, marks
//     the run start in a bitmap and sets its occupancy bits;
//   digits (strided): the run start below the digit from the bitmap, the
//     digit's plane index from it, its ADC value into the plane.
// A big window (more than kList digits, at most kMaxDig) keeps the plane
// index per run instead of per digit; a digit finds its run's number from the
// run starts counted before its bitmap word, and no digit list is made.
// Every read is bounds-checked against the segment counts from the headers and
// every write against the plane and the list.  Segment k may be empty.  Returns
// true (block-uniform) if every check passed.
struct WinSeg {
  const uint16_t* ent; const uint16_t* run; const uint32_t* adc;
  int ne, nrun, ndig, dfirst, tt_base, t_base_abs;
};

template <typename V>
__device__ __forceinline__ V sel3(int k, V a, V b, V c) { return k == 0 ? a : (k == 1 ? b : c); }

// (The three segments are separate by-value parameters: indexing an array of
// them with a runtime segment number would place it in local memory.)
__device__ __forceinline__ bool decode_window(const WinSeg s0, const WinSeg s1, const WinSeg s2, int np, int ps_stride,
                                              int nw, int T, const FindSmem& S, bool big) {
  const int tid = threadIdx.x, nt = (int)blockDim.x;
  const int ebase1 = s0.ne, ebase2 = s0.ne + s1.ne, ne = ebase2 + s2.ne;
  const int rbase1 = s0.nrun, rbase2 = s0.nrun + s1.nrun, nrun = rbase2 + s2.nrun;
  const int dbase1 = s0.ndig, dbase2 = s0.ndig + s1.ndig, ndig = dbase2 + s2.ndig;
  bool bad = ne > 2 * nt;
  // big window: run_L | run-start bitmap | run starts before each word, in the list area
  uint16_t* const runL = S.list;
  uint32_t* const dbmB = reinterpret_cast<uint32_t*>(S.list + kMaxRuns);
  uint16_t* const wpre = reinterpret_cast<uint16_t*>(dbmB + kBigWords);
  uint32_t* const dbm = big ? dbmB : S.dbm;
  if (big)
    for (int i = tid; i < kBigWords; i += nt) dbmB[i] = 0u;   // first read after the entries' barrier
  // ---- entries
  int e_t[2] = {0, 0}, e_nr[2] = {0, 0}, my_nr = 0;
#pragma unroll
  for (int j = 0; j < 2; j++) {
    const int e = 2 * tid + j;
    if (e >= ne || bad) continue;
    const int k = e < ebase1 ? 0 : (e < ebase2 ? 1 : 2);
    const int el = e - (k == 0 ? 0 : (k == 1 ? ebase1 : ebase2));
    const uint16_t* ent = sel3(k, s0.ent, s1.ent, s2.ent);
    const uint32_t v = ent[el];
    const int t_in = v & 0xff, nr = v >> 8, tt = t_in + sel3(k, s0.tt_base, s1.tt_base, s2.tt_base);
    if (nr < 1 || tt < 0 || tt >= kWinT || sel3(k, s0.t_base_abs, s1.t_base_abs, s2.t_base_abs) + t_in >= T) {
      bad = true;
      continue;
    }
    if (el > 0 && (int)(ent[el - 1] & 0xff) >= t_in) bad = true;   // strictly increasing t
    e_t[j] = t_in;
    e_nr[j] = nr;
    my_nr += nr;
  }
  uint32_t tot;
  const int r_first = (int)block_excl_scan32((uint32_t)my_nr, reinterpret_cast<uint32_t*>(S.scan), &tot);
  if ((int)tot != nrun) bad = true;
  {
    int r = r_first;
#pragma unroll
    for (int j = 0; j < 2; j++) {
      const int e = 2 * tid + j;
      if (e >= ne) continue;
      // a segment's first entry must start at the segment's first run
      if ((e == ebase1 && s1.ne > 0 && r != rbase1) || (e == ebase2 && s2.ne > 0 && r != rbase2)) bad = true;
      for (int q = 0; q < e_nr[j]; q++)
        if (r + q < kMaxRuns) S.run_t[r + q] = (uint8_t)e_t[j];
      r += e_nr[j];
    }
  }
  __syncthreads();
  // ---- runs
  const int per = (nrun + nt - 1) / nt;
  const int ra = min(tid * per, nrun), rb = min(ra + per, nrun);
  int my_nd = 0;
  for (int r = ra; r < rb; r++) {
    const int k = r < rbase1 ? 0 : (r < rbase2 ? 1 : 2);
    const int rl = r - (k == 0 ? 0 : (k == 1 ? rbase1 : rbase2));
    const uint16_t* run = sel3(k, s0.run, s1.run, s2.run);
    const uint32_t rv = run[rl];
    const int ps = rv & 0xff, len = rv >> 8;
    if (len < 1 || ps + len > np) { bad = true; continue; }
    if (rl > 0 && S.run_t[r - 1] == S.run_t[r]) {   // same time bin: ascending, disjoint
      const uint32_t pv = run[rl - 1];
      if (ps < (int)(pv & 0xff) + (int)(pv >> 8)) bad = true;
    }
    my_nd += len;
  }
  const int d_first = (int)block_excl_scan32((uint32_t)my_nd, reinterpret_cast<uint32_t*>(S.scan) + 20, &tot);
  if ((int)tot != ndig) bad = true;
  {
    int d = d_first;
    for (int r = ra; r < rb; r++) {
      const int k = r < rbase1 ? 0 : (r < rbase2 ? 1 : 2);
      const int rl = r - (k == 0 ? 0 : (k == 1 ? rbase1 : rbase2));
      const uint32_t rv = sel3(k, s0.run, s1.run, s2.run)[rl];
      const int ps = rv & 0xff, len = rv >> 8;
      if (len < 1 || ps + len > np) continue;
      // a segment's first run must start at the segment's first digit
      if ((r == rbase1 && s1.nrun > 0 && d != dbase1) || (r == rbase2 && s2.nrun > 0 && d != dbase2)) bad = true;
      const int tt = S.run_t[r] + sel3(k, s0.tt_base, s1.tt_base, s2.tt_base);   // stale if its entry failed: checked
      if (d + len <= ndig && d + len <= (big ? kMaxDig : kList) && tt >= 0 && tt < kWinT && r < kMaxRuns) {
        const uint16_t L0 = (uint16_t)(tt * ps_stride + kPad + ps);
        if (big) runL[r] = L0; else S.list[d] = L0;
        atomicOr(&dbm[d >> 5], 1u << (d & 31));
        set_occ(S, nw, tt, ps, len);
      } else {
        bad = true;
      }
      d += len;
    }
  }
  const bool valid = !__syncthreads_or(bad);
  if (!valid) return false;
  if (big) {
    // run starts before each bitmap word (run r starts at the r-th set bit)
    const int nwd = (ndig + 31) >> 5;
    const int per = (nwd + nt - 1) / nt;
    const int wa = min(tid * per, nwd), wb = min(wa + per, nwd);
    uint32_t c = 0;
    for (int i = wa; i < wb; i++) c += __popc(dbmB[i]);
    uint32_t tot3;
    uint32_t pre = block_excl_scan32(c, reinterpret_cast<uint32_t*>(S.scan), &tot3);
    for (int i = wa; i < wb; i++) {
      wpre[i] = (uint16_t)pre;
      pre += __popc(dbmB[i]);
    }
    __syncthreads();
  }
  // ---- digits
  const int nplane = kWinT * ps_stride;
  for (int d = tid; d < ndig; d += nt) {
    int w = d >> 5;
    uint32_t m = dbm[w] & (0xffffffffu >> (31 - (d & 31)));
    int L;
    if (big) {
      const int rr = min(max((int)wpre[w] + __popc(m) - 1, 0), kMaxRuns - 1);   // the run holding digit d
      while (m == 0 && w > 0) m = dbmB[--w];          // digit 0 always starts a run
      const int st = 32 * w + 31 - __clz(m);
      L = (int)runL[rr] + (d - st);
    } else {
      while (m == 0 && w > 0) m = S.dbm[--w];   // digit 0 always starts a run
      const int st = 32 * w + 31 - __clz(m);
      L = (int)S.list[st] + (d - st);
      if (d != st) S.list[d] = (uint16_t)L;
    }
    const int k = d < dbase1 ? 0 : (d < dbase2 ? 1 : 2);
    const int idx = sel3(k, s0.dfirst, s1.dfirst, s2.dfirst) + d - (k == 0 ? 0 : (k == 1 ? dbase1 : dbase2));
    const uint32_t word = sel3(k, s0.adc, s1.adc, s2.adc)[idx / 3];
    if (L < nplane) S.plane[L] = (uint16_t)((word >> (10 * (idx % 3))) & 1023u);
  }
  return true;
}

// Copy the byte range [a, b) of a page (2-byte aligned, both in bounds) to dst
// as 16-bit words, by one warp.
__device__ __forceinline__ void copy_u16_warp(uint16_t* dst, const uint8_t* pg, uint32_t a, uint32_t b) {
  const uint16_t* src = reinterpret_cast<const uint16_t*>(pg + a);
  for (uint32_t i = threadIdx.x & 31; i < (b - a) / 2; i += 32) dst[i] = __ldg(src + i);
}

// Peak test of the digit at plane index L (row tt, pad p): neighbours with a
// lower linear index (t * npads + p) must be strictly lower in charge, those
// with a higher index lower or equal; padding pads and empty pixels read 0.
__device__ __forceinline__ bool peak_at(const uint16_t* pl, int L, int ps_stride, int qmin) {
  const int q = pl[L];
  const uint16_t* u = pl + L - ps_stride;
  const uint16_t* d = pl + L + ps_stride;
  const int lo = max(max((int)u[-1], (int)u[0]), max((int)u[1], (int)pl[L - 1]));
  const int hi = max(max((int)pl[L + 1], (int)d[-1]), max((int)d[0], (int)d[1]));
  return (q >= qmin) & (q > lo) & (q >= hi);
}

// Index of the last prefix entry <= r in pre[0..n] (pre ascending, pre[0] = 0).
__device__ __forceinline__ int rank_search(const uint16_t* pre, int n, int r) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int)pre[mid] <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Five bits of a bitmap row around pad p: bit k <-> pad p - 2 + k (0 outside).
__device__ __forceinline__ uint32_t bits5(const uint32_t* row, int nw, int p) {
  const int lo = p - 2;                       // >= -2
  const int w0 = (lo + 32) / 32 - 1;          // floor(lo / 32)
  const uint32_t a = (w0 >= 0 && w0 < nw) ? row[w0] : 0u;
  const uint32_t b = (w0 + 1 >= 0 && w0 + 1 < nw) ? row[w0 + 1] : 0u;
  const unsigned long long v = ((unsigned long long)b << 32) | a;
  return (uint32_t)(v >> (lo - 32 * w0)) & 31u;
}

// Step 2b, 5x5 noise suppression of the peak at (tt, p): dropped when a peak
// of step 2 with a greater key lies on the ring of its 5x5 window and the
// pixel between the two (the inner pixel of the cluster rule toward it) lies
// less than min_dip ADC below the peak.  Reads the step-2 peak bitmap only.
__device__ __forceinline__ bool ns_drop(const FindSmem& S, int ps_stride, int nw, int tt, int p, int min_dip) {
  const uint16_t* c = S.plane + tt * ps_stride + kPad + p;
  const int qc = c[0];
#pragma unroll
  for (int dt = -2; dt <= 2; dt++) {
    uint32_t b = bits5(S.pk + (tt + dt) * nw, nw, p);
    if (dt > -2 && dt < 2) b &= 0x11u;        // rows -1..1: the pads at distance 2 only
    while (b) {
      const int dp = __ffs(b) - 3;
      b &= b - 1;
      const int qn = c[dt * ps_stride + dp];
      // greater key: more charge, or equal charge and a lower (t, p) index
      if (qn < qc || (qn == qc && (dt > 0 || (dt == 0 && dp > 0)))) continue;
      const int it = dt > 0 ? 1 : (dt < 0 ? -1 : 0), ip = dp > 0 ? 1 : (dp < 0 ? -1 : 0);
      if (qc - (int)c[it * ps_stride + ip] < min_dip) return true;
    }
  }
  return false;
}

// Cluster of the peak at (tt, p) of the window in shared memory: the 5x5 from
// the plane, the other peaks from the peak bitmap.
__device__ __forceinline__ void make_cluster(const FindSmem& S, int ps_stride, int nw, int np, int T, int s, int r,
                                             int f, int tt, int p, int xrow, uint4& rec, int4& xyz) {
  const uint16_t* c = S.plane + tt * ps_stride + kPad + p;
  int q[5][5];
#pragma unroll
  for (int dt = 0; dt < 5; dt++)
#pragma unroll
    for (int dp = 0; dp < 5; dp++) q[dt][dp] = c[(dt - 2) * ps_stride + dp - 2];
  uint32_t other = 0;
#pragma unroll
  for (int dt = -2; dt <= 2; dt++) {
    uint32_t b = bits5(S.pk + (tt + dt) * nw, nw, p);
    if (dt == 0) b &= ~4u;
    other |= b;
  }
  cluster_record(q, other != 0, np, T, s, r, f, tt, p, xrow, rec, xyz);
}

// L2 prefetch of the next window's input while the current one is being
// processed.  Fused finder and decode pass: its page and both neighbours,
// contiguous in the usual layout (at most 64 KB).  Find pass of the dense
// variant: its 262 plane rows, contiguous in the dense plane.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned long long n) {
  n = min(n, 65536ull) & ~15ull;
  if (n) {
    const size_t ga = __cvta_generic_to_global(p);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ga), "r"((unsigned)n) : "memory");
  }
}

__device__ __forceinline__ void prefetch_next_pages(const DevWork& W, const unsigned long long (&noffs)[4]) {
  const unsigned long long lo = noffs[0] != ~0ull ? noffs[0] : noffs[1];
  unsigned long long hi = noffs[3] != ~0ull ? noffs[3] : W.pages_bytes;
  if (lo < hi && lo < W.pages_bytes && (lo & 15) == 0)
    prefetch_l2(W.pages + lo, min(hi, (unsigned long long)W.pages_bytes) - lo);
}

__device__ __forceinline__ void prefetch_next_dense(const DevGeom& G, const DevWork& W, unsigned nt) {
  const unsigned sr = nt / (unsigned)G.n_frag, f = nt - sr * (unsigned)G.n_frag;
  const long long T = G.n_time_bins;
  const long long t0 = max(0ll, (long long)kFrag * f - kHalo), t1 = min(T, (long long)kFrag * (f + 1) + kHalo);
  if (t0 >= t1) return;
  const size_t row = (size_t)W.dense_stride * 2;   // bytes, a multiple of 16
  const uint8_t* base = reinterpret_cast<const uint8_t*>(W.dense) + ((size_t)sr * T + t0) * row;
  const unsigned long long n = (unsigned long long)(t1 - t0) * row;
  prefetch_l2(base, n);
  if (n > 65536ull) prefetch_l2(base + 65536, n - 65536ull);
}

// Output modes.  kScratch (the pipeline): each window reserves a span of the
// scratch buffer with one atomic and writes its records there; a scan over the
// window counts and k_compact_clusters then place them in canonical order and
// derive the per-cluster (X, Y, Z, t_peak) arrays.  No window waits for
// another.  Otherwise (the allocation-free entry point, which has no scratch
// buffer for records): a decoupled look-back over the windows gives each its
// canonical offset and the records are written in place; only the records.
// The neighbour pages' 32-byte headers of a window into hdr[0..3] (two 16-byte
// halves of the previous page, then of the next page), zero where the window
// has no such neighbour or the offset is unusable; plain loads, or 16-byte
// cp.async copies (one group, committed) that the caller waits for before use.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(__cvta_generic_to_global(src)) : "memory");
}

template <int kMode, bool kAsync>
__device__ __forceinline__ void load_nb_headers(const DevGeom& G, const DevWork& W, int frs, uint64_t op, uint64_t on,
                                                uint4* hdr);

// The next window (index in S.misc[1], coordinates in S.misc[2], its page
// offsets in S.offs): its three pages prefetched into L2, its neighbours'
// headers copied into shared memory.
template <int kMode>
__device__ __forceinline__ void issue_next(const DevGeom& G, const DevWork& W, const FindSmem& S,
                                           unsigned int n_windows) {
  if ((unsigned)S.misc[1] >= n_windows) return;
  const unsigned long long no[4] = {S.offs[0], S.offs[1], S.offs[2], S.offs[3]};
  prefetch_next_pages(W, no);
  load_nb_headers<kMode, true>(G, W, S.misc[2], no[0], no[2], S.hdr);
}

template <int kMode, bool kAsync>
__device__ __forceinline__ void load_nb_headers(const DevGeom& G, const DevWork& W, int frs, uint64_t op, uint64_t on,
                                                uint4* hdr) {
  const int f = frs & 0xffff;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const uint64_t o2 = k < 2 ? op : on;
    const bool want = kMode == 0 && (k < 2 ? f > 0 : f + 1 < G.n_frag) && o2 != ~0ull && (o2 & 15) == 0 &&
                      o2 <= W.pages_bytes && W.pages_bytes - o2 >= 32;
    const uint4* src = reinterpret_cast<const uint4*>(W.pages + (want ? o2 : 0)) + (k & 1);
    if (!want) hdr[k] = make_uint4(0u, 0u, 0u, 0u);
    else if (kAsync) cp_async16(hdr + k, src);
    else hdr[k] = __ldg(src);
  }
  if (kAsync) asm volatile("cp.async.commit_group;" ::: "memory");
}

// kMode: 0 the fused finder (pages -> clusters); 1 and 2 the dense-plane
// variant: 1 decodes each window's own page into a dense HBM plane of ADC
// values, 2 reads a window and its 3-bin halos back from that plane and runs
// the same peak / cluster steps.  All three give the same clusters.  kNs:
// step 2b (5x5 noise suppression) compiled in, for ns_min_dip > 0.
template <bool kScratch, int kThreads, int kMode, bool kNs>
__global__ void __launch_bounds__(kThreads, 2)
k_find_clusters(DevGeom G, DevParams P, DevWork W, unsigned int n_windows) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ps_stride = G.npmax + 2 * kPad, nw = G.nw;
  const int nown_words = kFrag * nw;         // plane rows 3 .. 258
  const int nplane = kWinT * ps_stride;
  const bool use_list = nplane <= 65536;     // plane indices fit the 16-bit lists
  const uint32_t magic = (uint32_t)((0x100000000ull + ps_stride - 1) / ps_stride);  // row = umulhi(L, magic)
  FindSmem S;
  {
    size_t o = 0;
    S.plane = reinterpret_cast<uint16_t*>(smem_raw + o);
    o += ((size_t)nplane * 2 + 15) & ~(size_t)15;
    S.occ = reinterpret_cast<uint32_t*>(smem_raw + o);
    o += (size_t)kWinT * nw * 4;
    S.pk = reinterpret_cast<uint32_t*>(smem_raw + o);
    o += (size_t)kWinT * nw * 4;
    S.dbm = reinterpret_cast<uint32_t*>(smem_raw + o);
    o += (size_t)kRunMapWords * 4;
    o = (o + 15) & ~(size_t)15;
    S.st_rec = reinterpret_cast<uint4*>(smem_raw + o);
    o += kStage * 16;
    S.st_xyz = reinterpret_cast<int4*>(smem_raw + o);
    o += kStage * 16;
    S.plist = reinterpret_cast<uint16_t*>(smem_raw + o);
    o += kStage * 2;
    S.ppre = reinterpret_cast<uint16_t*>(smem_raw + o);
    o += ((size_t)nown_words + 1) * 2;
    o = (o + 15) & ~(size_t)15;
    S.halo = smem_raw + o;
    o += 2 * kHaloStage;
    S.hdr = reinterpret_cast<uint4*>(smem_raw + o);
    o += 4 * 16;
    S.offs = reinterpret_cast<unsigned long long*>(smem_raw + o);
    o += 4 * 8;
    S.scan = reinterpret_cast<unsigned long long*>(smem_raw + o);
    o += 34 * 8;
    S.misc = reinterpret_cast<int32_t*>(smem_raw + o);
    o += 16 * 4;
    S.ph = reinterpret_cast<PageHdr*>(smem_raw + o);
    o += 3 * sizeof(PageHdr);
    o = (o + 15) & ~(size_t)15;
    S.list = reinterpret_cast<uint16_t*>(smem_raw + o);
    o += kList * 2;
    S.run_t = reinterpret_cast<uint8_t*>(smem_raw + o);
    o += kMaxRuns;
  }
  const int tid = threadIdx.x;
  const int opt = (nown_words + blockDim.x - 1) / blockDim.x;
  uint8_t* own_stage = reinterpret_cast<uint8_t*>(S.st_rec);
  const uint32_t own_stage_bytes = (uint32_t)(((size_t)2 * kStage * 16 + kStage * 2 + ((size_t)nown_words + 1) * 2) & ~(size_t)15);

  if (kScratch && blockIdx.x == 0 && tid == 0) W.ctr[CTR_NWIN] = n_windows;
  // the plane starts empty and is kept empty between windows
  for (int i = tid; i < nplane / 2; i += blockDim.x) reinterpret_cast<uint32_t*>(S.plane)[i] = 0u;
  if (tid == 0 && (nplane & 1)) S.plane[nplane - 1] = 0;

  // With scratch output no window waits for another, so the next window is
  // taken early: its ticket at the top of the current one, its page offsets
  // after the decode, and its three-page byte range is prefetched into L2
  // after the peak test.  In look-back mode a held window would stall every
  // successor's look-back: there the ticket is taken only at the top.
  // windows of this kernel: all, or (with the light path) the heavy list
  const unsigned long long n_heavy = (kScratch && W.heavy_list) ? W.ctr[CTR_NHEAVY] : 0ull;
  auto window_of = [&](unsigned tk) -> unsigned {
    if constexpr (!kScratch) {
      return tk;
    } else {
      if (!W.heavy_list) return tk;
      return (unsigned long long)tk < n_heavy ? W.heavy_list[tk] : n_windows;
    }
  };
  if (kScratch && tid == 0) {
    const unsigned w0 = window_of(atomicAdd(&W.tickets[kMode == 2 ? TK_FIND2 : TK_FIND], 1u));
    S.misc[1] = (int)w0;
    S.misc[2] = w0 < n_windows ? window_frs(G, w0) : 0;
    for (int k = 0; k < 4; k++) {
      const long long j = (long long)w0 - 1 + k;
      S.offs[k] = (j >= 0 && j < (long long)n_windows && w0 < n_windows) ? W.page_offsets[j] : ~0ull;
    }
    if (kMode != 2 && w0 < n_windows) load_nb_headers<kMode, false>(G, W, S.misc[2], S.offs[0], S.offs[2], S.hdr);
  }
  unsigned int nt = 0;                  // next window (thread 0, scratch mode)
  // the thread that prefetches the next window and copies its neighbours'
  // headers (cp.async groups belong to the issuing thread, which also waits):
  // the last one in the fused finder, idle while the first threads build the
  // clusters; thread 0 in the dense variant's decode pass
  const int issuer = kMode == 0 ? (int)blockDim.x - 1 : 0;
  while (true) {
    // ---- 0. window w (scratch mode: its neighbours' headers were copied
    // during the previous window)
    if (!kScratch && tid == 0) {
      const unsigned wt = atomicAdd(&W.tickets[TK_FIND], 1u);
      S.misc[1] = (int)wt;
      S.misc[2] = wt < n_windows ? window_frs(G, wt) : 0;
    }
    if (kScratch && kMode != 2 && tid == issuer) asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const unsigned int w = (unsigned int)S.misc[1];
    if (w >= n_windows) break;
    if (kScratch && tid == 0) nt = window_of(atomicAdd(&W.tickets[kMode == 2 ? TK_FIND2 : TK_FIND], 1u));
    if (!kScratch && tid == 0) {
      for (int k = 0; k < 4; k++) {
        const long long j = (long long)w - 1 + k;
        S.offs[k] = (j >= 0 && j < (long long)n_windows) ? W.page_offsets[j] : ~0ull;
      }
      if (kMode != 2) load_nb_headers<kMode, false>(G, W, S.misc[2], S.offs[0], S.offs[2], S.hdr);
    }
    {
      // occ, pk and dbm are adjacent: clear them as 16-byte words (the tail word by word)
      const int nwords = 2 * kWinT * nw + kRunMapWords;
      uint4* o4 = reinterpret_cast<uint4*>(S.occ);
      for (int i = tid; i < nwords / 4; i += blockDim.x) o4[i] = make_uint4(0u, 0u, 0u, 0u);
      for (int i = (nwords & ~3) + tid; i < nwords; i += blockDim.x) S.occ[i] = 0u;
    }
    __syncthreads();
    const int frs = S.misc[2];
    const int f = frs & 0xffff, r = (frs >> 16) & 0xff, s = (frs >> 24) & 0xff;   // s: physical sector
    const int np = G.npads[r];
    const int T = G.n_time_bins;
    const uint64_t off = S.offs[1];

    bool ok;
    int ndig;
    bool listed;
    if (kMode != 2) {
      // ---- 1. one round trip: stage the page (length guessed from the next
      // page's offset); warps 0-2 copy the previous page's entries / runs / ADC
      // words of its last 3 bins, warps 3-5 the next page's of its first 3 bins
      // (the neighbours' headers are already in shared memory), warp 6 parses
      // the own header from global memory: all copies in flight together
      uint32_t copied = 0;
      if (off <= W.pages_bytes && W.pages_bytes - off >= 32 && (off & 15) == 0) {
        uint64_t guess = (S.offs[2] != ~0ull && S.offs[2] > off) ? S.offs[2] - off : W.pages_bytes - off;
        guess = min(guess, (uint64_t)own_stage_bytes);
        guess = min(guess, W.pages_bytes - off);
        copied = (uint32_t)(guess & ~15ull);
        const uint4* src = reinterpret_cast<const uint4*>(W.pages + off);
        for (uint32_t i = tid; i < copied / 16; i += blockDim.x) reinterpret_cast<uint4*>(own_stage)[i] = __ldg(src + i);
      }
      const bool own_global = copied < 32;
      {
        const int wid = tid >> 5, lane = tid & 31;
        if (wid < 6) {
          const int nb = wid < 3 ? 0 : 1;   // 0: previous page, 1: next page
          PageHdr hh;
          uint32_t a = 0, b = 0;
          int okk = 0;
          if (lane == 0) {
            const bool want = kMode != 1 && (nb == 0 ? f > 0 : f + 1 < G.n_frag);
            okk = want && parse_header(S.hdr + 2 * nb, S.offs[2 * nb], W.pages_bytes, hh);
            if (nb == 0)
              okk = okk && 2 * (hh.n_tb - hh.hi_tb) <= kHaloRunOff &&
                    2 * (hh.n_runs - hh.hi_runs) <= kHaloAdcOff - kHaloRunOff &&
                    4 * ((hh.n_dig + 2) / 3 - hh.hi_dig / 3) <= kHaloStage - kHaloAdcOff;
            else
              okk = okk && 2 * hh.lo_tb <= kHaloRunOff && 2 * hh.lo_runs <= kHaloAdcOff - kHaloRunOff &&
                    4 * ((hh.lo_dig + 2) / 3) <= kHaloStage - kHaloAdcOff;
            if (okk) {
              const int part = wid % 3;
              if (nb == 0) {
                if (part == 0) { a = 32 + 2 * hh.hi_tb; b = 32 + 2 * hh.n_tb; }
                else if (part == 1) { a = 32 + 2 * hh.n_tb + 2 * hh.hi_runs; b = 32 + 2 * hh.n_tb + 2 * hh.n_runs; }
                else { a = hh.body + 4 * (hh.hi_dig / 3); b = hh.body + 4 * ((hh.n_dig + 2) / 3); }
              } else {
                if (part == 0) { a = 32; b = 32 + 2 * hh.lo_tb; }
                else if (part == 1) { a = 32 + 2 * hh.n_tb; b = 32 + 2 * hh.n_tb + 2 * hh.lo_runs; }
                else { a = hh.body; b = hh.body + 4 * ((hh.lo_dig + 2) / 3); }
              }
            }
            if (wid == 0 || wid == 3) {
              S.ph[1 + nb] = hh;
              S.misc[5 + nb] = okk;
            }
          }
          okk = __shfl_sync(0xffffffffu, okk, 0);
          a = __shfl_sync(0xffffffffu, a, 0);
          b = __shfl_sync(0xffffffffu, b, 0);
          if (okk) {
            const int part = wid % 3;
            const int doff = part == 0 ? 0 : (part == 1 ? kHaloRunOff : kHaloAdcOff);
            copy_u16_warp(reinterpret_cast<uint16_t*>(S.halo + nb * kHaloStage + doff),
                          W.pages + S.offs[2 * nb], a, b);
          }
        } else if (wid == 6 && lane == 0) {
          PageHdr hh;
          const bool okk = parse_header(reinterpret_cast<const uint4*>(W.pages + off), off, W.pages_bytes, hh) &&
                           hh.sector == s && hh.row == r && hh.frag == f;
          S.ph[0] = hh;
          S.misc[4] = okk;
        }
      }
      __syncthreads();
      ok = S.misc[4];
      const bool okp = S.misc[5], okn = S.misc[6];
      const PageHdr& h = S.ph[0];
      const PageHdr& hp = S.ph[1];
      const PageHdr& hn = S.ph[2];
      const uint8_t* own = (own_global || h.len > copied) ? W.pages + off : own_stage;
      uint8_t* hprev = S.halo;
      uint8_t* hnext = S.halo + kHaloStage;

      // ---- 3. decode the own page (block) and the two halos (the last two warps,
      // while the others write the own digits); digits listed as own | previous
      // halo | next halo
      const int n_own = ok ? h.n_dig : 0;
      const int n_prev = okp ? hp.n_dig - hp.hi_dig : 0;
      const int n_next = okn ? hn.lo_dig : 0;
      ndig = n_own + n_prev + n_next;
      listed = use_list && ndig <= kList;
      {
        const Seg gp{reinterpret_cast<const uint16_t*>(hprev), hp.n_tb - hp.hi_tb,
                     reinterpret_cast<const uint16_t*>(hprev + kHaloRunOff), hp.n_runs - hp.hi_runs,
                     reinterpret_cast<const uint32_t*>(hprev + kHaloAdcOff), hp.hi_dig % 3, n_prev,
                     kHalo - kFrag, kFrag * (f - 1), listed ? n_own : kList, false};
        const Seg gn{reinterpret_cast<const uint16_t*>(hnext), hn.lo_tb,
                     reinterpret_cast<const uint16_t*>(hnext + kHaloRunOff), hn.lo_runs,
                     reinterpret_cast<const uint32_t*>(hnext + kHaloAdcOff), 0, n_next, kHalo + kFrag, kFrag * (f + 1),
                     listed ? n_own + n_prev : kList, false};
        const Seg go{reinterpret_cast<const uint16_t*>(own + 32), h.n_tb,
                     reinterpret_cast<const uint16_t*>(own + 32 + 2 * h.n_tb), h.n_runs,
                     reinterpret_cast<const uint32_t*>(own + h.body), 0, h.n_dig, kHalo, kFrag * f,
                     listed ? 0 : kList, true};
        const int nrun_all = (okp ? hp.n_runs - hp.hi_runs : 0) + (ok ? h.n_runs : 0) + (okn ? hn.lo_runs : 0);
        if (ok && use_list && nrun_all <= kMaxRuns && ndig <= kMaxDig) {
          const WinSeg s0{gp.ent, gp.run, gp.adc, okp ? gp.ne : 0, okp ? gp.nrun : 0, n_prev, gp.dfirst, gp.tt_base,
                          gp.t_base_abs};
          const WinSeg s1{go.ent, go.run, go.adc, go.ne, go.nrun, n_own, 0, go.tt_base, go.t_base_abs};
          const WinSeg s2{gn.ent, gn.run, gn.adc, okn ? gn.ne : 0, okn ? gn.nrun : 0, n_next, 0, gn.tt_base,
                          gn.t_base_abs};
          ok = decode_window(s0, s1, s2, np, ps_stride, nw, T, S, !listed);
        } else {
          ok = decode_seg(go, ok, np, ps_stride, nw, T, S, okp ? &gp : nullptr, okn ? &gn : nullptr);
        }
      }
      if (!ok && tid == 0) atomicOr(W.err, kErrCorrupt);
      __syncthreads();
    } else {
      // ---- 1-3 (dense variant): rows t0-3 .. t0+258 of the dense plane, as
      // 16-byte chunks of 8 pads (a warp-uniform loop, kDenseU chunks a thread
      // in flight), into the shared plane with their occupancy bits; the digit
      // list is filled in the same pass.  Its order is free (the peak test and
      // the clearing do not depend on it): a warp scan of the chunks' digit
      // counts and one shared atomic per warp and round give the slots.
      const int sr = (int)(w / (unsigned)G.n_frag);
      const size_t rbase = (size_t)sr * T;
      const int cpr = (int)(W.dense_stride >> 3);
      const int nitems = kWinT * cpr;
      const uint4* dsrc = reinterpret_cast<const uint4*>(W.dense);
      const int lane = tid & 31;
      if (tid == 0) S.misc[8] = 0;
      __syncthreads();
      const uint32_t cmagic = (uint32_t)((0x100000000ull + cpr - 1) / cpr);   // i / cpr = umulhi(i, cmagic)
      for (int i0 = tid - lane; i0 < nitems; i0 += kDenseU * (int)blockDim.x) {
        uint4 v[kDenseU];
#pragma unroll
        for (int u = 0; u < kDenseU; u++) {
          const int i = i0 + u * (int)blockDim.x + lane;
          v[u] = make_uint4(0u, 0u, 0u, 0u);
          if (i < nitems) {
            const int tt = (int)__umulhi((uint32_t)i, cmagic), c = i - tt * cpr;
            const int t = kFrag * f + tt - kHalo;
            if (t >= 0 && t < T) v[u] = __ldg(dsrc + (rbase + t) * cpr + c);
          }
        }
        // plane and occupancy; the chunks' digit bits kept for the list
        unsigned long long bits = 0;
        int n = 0;
#pragma unroll
        for (int u = 0; u < kDenseU; u++) {
          const uint32_t wv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
          if (wv[0] | wv[1] | wv[2] | wv[3]) {   // most chunks are empty
            const int i = i0 + u * (int)blockDim.x + lane;
            const int tt = (int)__umulhi((uint32_t)i, cmagic), c = i - tt * cpr;
            const int L0 = tt * ps_stride + kPad + 8 * c;
            uint32_t bits8 = 0;
#pragma unroll
            for (int j = 0; j < 8; j++) {
              const uint16_t q = (uint16_t)(wv[j >> 1] >> (16 * (j & 1)));
              if (q && 8 * c + j < np) {
                S.plane[L0 + j] = q;
                bits8 |= 1u << j;
              }
            }
            if (bits8) atomicOr(&S.occ[tt * nw + ((8 * c) >> 5)], bits8 << ((8 * c) & 31));
            bits |= (unsigned long long)bits8 << (8 * u);
            n += __popc(bits8);
          }
        }
        // list slots: a warp scan of the threads' digit counts, one atomic a warp
        int incl = n;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += y;
        }
        int base = 0;
        if (lane == 31 && incl) base = atomicAdd(&S.misc[8], incl);
        base = __shfl_sync(0xffffffffu, base, 31);
        int k = base + incl - n;
        while (bits) {
          const int bpos = __ffsll((long long)bits) - 1;
          bits &= bits - 1;
          const int u = bpos >> 3, j = bpos & 7;
          const int i = i0 + u * (int)blockDim.x + lane;
          const int tt = (int)__umulhi((uint32_t)i, cmagic), c = i - tt * cpr;
          if (use_list && k < kList) S.list[k] = (uint16_t)(tt * ps_stride + kPad + 8 * c + j);
          k++;
        }
      }
      __syncthreads();
      ndig = S.misc[8];
      listed = use_list && ndig <= kList;
      ok = true;
      __syncthreads();
    }

    if (kScratch && tid == 0) {
      // the next window's index, coordinates and page offsets (this window
      // reads neither S.misc[1..2] nor S.offs any more)
      S.misc[1] = (int)nt;
      S.misc[2] = nt < n_windows ? window_frs(G, nt) : 0;
      for (int k = 0; k < 4; k++) {
        const long long j = (long long)nt - 1 + k;
        S.offs[k] = (nt < n_windows && j >= 0 && j < (long long)n_windows) ? W.page_offsets[j] : ~0ull;
      }
    }

    if (kMode == 1) {
      if (kScratch && tid == issuer) issue_next<kMode>(G, W, S, n_windows);
      // ---- dense variant, decode pass: the window's own rows into the dense
      // plane, 16-byte chunks of 8 pads (pads past the row's end written as 0)
      const int sr = (int)(w / (unsigned)G.n_frag);
      const int nrows = min(kFrag, T - kFrag * f);
      const int cpr = (int)(W.dense_stride >> 3);
      uint4* ddst = reinterpret_cast<uint4*>(W.dense) + ((size_t)sr * T + (size_t)kFrag * f) * cpr;
      for (int i = tid; i < nrows * cpr; i += blockDim.x) {
        const int q = i / cpr, c = i - q * cpr;
        const uint16_t* src = S.plane + (q + kHalo) * ps_stride + kPad + 8 * c;
        uint32_t wv[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const uint32_t lo = 8 * c + 2 * j < np ? src[2 * j] : 0u;
          const uint32_t hi = 8 * c + 2 * j + 1 < np ? src[2 * j + 1] : 0u;
          wv[j] = lo | (hi << 16);
        }
        ddst[i] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
      }
      __syncthreads();
    } else {
      // ---- 4. peak test, one digit per thread (rows 1..260; rows 0 and 261 only
      // serve as neighbours)
      if (ok) {
        if (listed) {
          for (int i = tid; i < ndig; i += blockDim.x) {
            const int L = S.list[i];
            if (L >= nplane) continue;
            const int tt = (int)__umulhi((uint32_t)L, magic);
            if (tt < 1 || tt > kWinT - 2) continue;
            if (peak_at(S.plane, L, ps_stride, P.q_peak_min)) {
              const int p = L - tt * ps_stride - kPad;
              atomicOr(&S.pk[tt * nw + (p >> 5)], 1u << (p & 31));
            }
          }
        } else {
          // too many digits to list: the occupied pixels of rows 1..260 in
          // equal shares per thread; a scan of the occupancy words' counts,
          // kept in the (now free) list area, finds each share's first word
          const int w0 = nw, nwd = (kWinT - 2) * nw;
          uint16_t* const wpre = S.list;
          const int per = (nwd + (int)blockDim.x - 1) / (int)blockDim.x;
          const int a = min(tid * per, nwd), b = min(a + per, nwd);
          uint32_t c = 0;
          for (int i = a; i < b; i++) c += __popc(S.occ[w0 + i]);
          uint32_t tot;
          uint32_t pre = block_excl_scan32(c, reinterpret_cast<uint32_t*>(S.scan), &tot);
          for (int i = a; i < b; i++) {
            wpre[i] = (uint16_t)pre;
            pre += __popc(S.occ[w0 + i]);
          }
          __syncthreads();
          if (tot <= 65535u) {
            const uint32_t share = (tot + blockDim.x - 1) / blockDim.x;
            const uint32_t k0 = min(tid * share, tot), k1 = min(k0 + share, tot);
            if (k0 < k1) {
              int lo = 0, hi = nwd - 1;   // the last word whose count prefix is <= k0
              while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((uint32_t)wpre[mid] <= k0) lo = mid; else hi = mid - 1;
              }
              int wi = lo;
              uint32_t word = S.occ[w0 + wi];
              for (uint32_t q = k0 - wpre[wi]; q > 0; q--) word &= word - 1;
              for (uint32_t k = k0; k < k1; k++) {
                while (word == 0 && wi + 1 < nwd) word = S.occ[w0 + ++wi];
                if (word == 0) break;
                const int bb = __ffs(word) - 1;
                word &= word - 1;
                const int gw = w0 + wi, tt = gw / nw, p0 = (gw % nw) * 32;
                if (peak_at(S.plane, tt * ps_stride + kPad + p0 + bb, ps_stride, P.q_peak_min))
                  atomicOr(&S.pk[gw], 1u << bb);
              }
            }
          } else {   // more than 2^16 occupied pixels: word by word
            for (int wi_ = nw + tid; wi_ < (kWinT - 1) * nw; wi_ += blockDim.x) {
              uint32_t word = S.occ[wi_];
              const int tt = wi_ / nw, p0 = (wi_ % nw) * 32;
              while (word) {
                const int bq = __ffs(word) - 1;
                word &= word - 1;
                if (peak_at(S.plane, tt * ps_stride + kPad + p0 + bq, ps_stride, P.q_peak_min))
                  atomicOr(&S.pk[wi_], 1u << bq);
              }
            }
          }
        }
      }
      __syncthreads();

      // ---- 4b. noise suppression (optional): the surviving own peaks go to
      // the own rows of the occupancy bitmap, which afterwards only serves to
      // clear the plane of an unlisted window (then cleared whole instead)
      if (kNs) {
        for (int i = tid; i < nown_words; i += blockDim.x) {
          uint32_t word = S.pk[kHalo * nw + i], keep = word;
          const int tt = kHalo + i / nw, p0 = (i % nw) * 32;
          while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            if (ns_drop(S, ps_stride, nw, tt, p0 + b, P.ns_min_dip)) keep &= ~(1u << b);
          }
          S.occ[kHalo * nw + i] = keep;
        }
        __syncthreads();
      }
      // the own peaks that become clusters (rows 3..258)
      const uint32_t* const sv = (kNs ? S.occ : S.pk) + kHalo * nw;

      if (kMode == 2 && kScratch && tid == 0 && nt < n_windows) prefetch_next_dense(G, W, nt);

      // ---- 5. rank the own peaks (rows 3..258) in canonical order, list the
      // first kStage, publish the window's count
      int npk;
      {
        const int w0 = tid * opt, w1 = min(w0 + opt, nown_words);
        int c = 0;
        for (int i = w0; i < w1; i++) c += __popc(sv[i]);
        uint32_t tot;
        const uint32_t pre = block_excl_scan32((uint32_t)c, reinterpret_cast<uint32_t*>(S.scan), &tot);
        int run = (int)pre;
        for (int i = w0; i < w1; i++) {
          uint32_t word = sv[i];
          S.ppre[i] = (uint16_t)run;
          while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            if (run < kStage && use_list) {
              const int wi_ = i + kHalo * nw;
              S.plist[run] = (uint16_t)((wi_ / nw) * ps_stride + kPad + (wi_ % nw) * 32 + b);
            }
            run++;
          }
        }
        if (tid == 0) {
          S.ppre[nown_words] = (uint16_t)tot;
          if (!kScratch) lookback_publish(W.win_state, (long long)w, tot);
        }
        npk = (int)tot;
      }
      __syncthreads();

      if (kMode == 0 && kScratch && tid == issuer) issue_next<kMode>(G, W, S, n_windows);

      // ---- 6. clusters of the first kStage peaks, one thread each, staged
      const int nst = min(npk, kStage);
      for (int k = tid; k < nst; k += blockDim.x) {
        int tt, p;
        if (use_list) {
          const int L = S.plist[k];
          tt = (int)__umulhi((uint32_t)L, magic);
          p = L - tt * ps_stride - kPad;
        } else {   // rows too wide for 16-bit plane indices
          const int wo = rank_search(S.ppre, nown_words + 1, k);
          tt = kHalo + wo / nw;
          p = (wo % nw) * 32 + __fns(sv[wo], 0, k - (int)S.ppre[wo] + 1);
        }
        make_cluster(S, ps_stride, nw, np, T, s, r, f, tt, p, G.xrow[r], S.st_rec[k], S.st_xyz[k]);
      }

      // ---- 7. where the records go: a scratch span (one atomic) or, without
      // scratch, the canonical offset from the decoupled look-back
      if (kScratch) {
        if (tid == 0) {
          const unsigned long long so = atomicAdd(&W.ctr[CTR_SCURSOR], (unsigned long long)npk);
          if (so + npk > W.cap_cl) atomicOr(W.err, kErrOverflowCl);
          W.win_cnt[w] = (unsigned long long)npk;
          W.win_soff[w] = (uint32_t)min(so, (unsigned long long)W.cap_cl);
          S.scan[33] = so;
        }
      } else if (tid < 32) {
        const unsigned long long base = lookback_wait(W.win_state, (long long)w, (unsigned long long)npk, W.err);
        if (tid == 0) {
          S.scan[33] = base;
          if (w == n_windows - 1) W.ctr[CTR_NCL] = base + npk;
          if (base + npk > W.cap_cl) atomicOr(W.err, kErrOverflowCl);
        }
      }
      __syncthreads();
      const unsigned long long base = S.scan[33];
      tpc_cluster* const dst = kScratch ? W.scratch_cl : W.clusters;

      // ---- 8. write out: staged records coalesced, any beyond one thread each
      for (int k = tid; k < npk; k += blockDim.x) {
        const unsigned long long idx = base + k;
        if (idx >= W.cap_cl) break;   // overflow: keep [0, cap) free of gaps, drop the rest
        uint4 rec;
        int4 xyz;
        if (k < kStage) {
          rec = S.st_rec[k];
        } else {
          const int wo = rank_search(S.ppre, nown_words + 1, k);
          const int bit = __fns(sv[wo], 0, k - (int)S.ppre[wo] + 1);
          make_cluster(S, ps_stride, nw, np, T, s, r, f, kHalo + wo / nw, (wo % nw) * 32 + bit, G.xrow[r], rec, xyz);
        }
        reinterpret_cast<uint4*>(dst)[idx] = rec;
      }
      __syncthreads();
    }

    // ---- 9. leave the plane empty for the next window
    if (listed) {
      for (int i = tid; i < ndig; i += blockDim.x) {
        const int L = S.list[i];
        if (L < nplane) S.plane[L] = 0;
      }
    } else {
      // an unlisted window is dense: clear the whole plane, 16 bytes a store
      // (balanced; with noise suppression occ's own rows no longer hold the digits)
      const int n16 = nplane / 8;
      for (int i = tid; i < n16; i += blockDim.x) reinterpret_cast<uint4*>(S.plane)[i] = make_uint4(0u, 0u, 0u, 0u);
      for (int i = 8 * n16 + tid; i < nplane; i += blockDim.x) S.plane[i] = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Light windows.  Half of a full-TPC timeframe's windows hold at most a few
// hundred digits (noise and the outer tracks), yet a window costs the block
// finder about 10 k cycles of fixed latency (round trips, block barriers,
// scans over its 74 KB plane).  Such a window (at most kLightDig digits and
// runs with its halos) is given to one warp instead: its digits are decoded
// from its page and halo ranges (staged in the warp's shared memory) into a
// per-warp list sorted by (plane row, pad) with each row's digit range, and
// the peak test and the 5x5 clusters look pixels up by scanning a row.  The
// results are those of the block path (the same rules, the same record
// builder).
constexpr int kLightDig = 256;               // digits (and runs) of a light window, halos included (384, 512: no faster)
constexpr int kLightWarps = 6;               // warps per light block
constexpr int kLightBlocksPerSm = 4;
constexpr unsigned kLightMinWindows = 4096;  // smaller timeframes: block finder only
// a light window's own page: header, <= 256 entries, <= kLightDig runs and digits
constexpr int kLightOwn = (32 + 2 * 256 + 2 * kLightDig + 4 * ((kLightDig + 2) / 3) + 15) / 16 * 16;
// a neighbour's halo: <= 3 entries | runs at byte 16 | ADC words at kHaloAdcAt
constexpr int kHaloAdcAt = 16 + 2 * kLightDig;
constexpr int kLightHalo = (kHaloAdcAt + 4 * (kLightDig / 3 + 2) + 15) / 16 * 16;

struct LightWarp {
  uint4 own[kLightOwn / 16];    // the own page, staged
  uint4 halo[2][kLightHalo / 16];   // the neighbours' halo entries / runs / ADC words, staged
  uint16_t row0[kWinT + 2];     // first digit of each plane row (digits are sorted by row, pad)
  uint16_t row1[kWinT + 2];     // one past its last
  uint16_t dt[kLightDig];       // plane row of digit d (0..261)
  uint16_t dq[kLightDig];       // its ADC value
  uint8_t dp[kLightDig];        // its pad
  uint8_t run_t[kLightDig];     // time bin (within its page) of run r
  uint32_t pk[kLightDig / 32];  // digit d is a peak of step 2
  uint32_t sv[kLightDig / 32];  // ... and survives step 2b (the clusters)
};

// Digit index of pixel (row tt, pad p) of the warp's window, or -1: a short
// scan of the row's digits (pads ascending).
__device__ __forceinline__ int light_find(const LightWarp& L, int tt, int p, int np) {
  if (p < 0 || p >= np || tt < 0 || tt >= kWinT) return -1;
  const int e = L.row1[tt];
  for (int i = L.row0[tt]; i < e; i++) {
    const int pi = L.dp[i];
    if (pi == p) return i;
    if (pi > p) break;
  }
  return -1;
}

__device__ __forceinline__ int light_q(const LightWarp& L, int tt, int p, int np) {
  const int i = light_find(L, tt, p, np);
  return i < 0 ? 0 : (int)L.dq[i];
}

// One segment of a light window: a page's entries / runs / digits in a range.
struct LightSeg {
  const uint16_t* ent;   // its first entry
  const uint16_t* run;   // its first run
  const uint32_t* adc;   // the page's ADC words
  int ne, nrun, ndig;    // counts in the segment
  int dfirst;            // page digit index of the segment's first digit
  int tt_base;           // plane row = t_in + tt_base
  int t_base;            // absolute time bin = t_in + t_base
};

// Classify the windows: light (one warp) or block.  A window is light when its
// own header and its neighbours' are valid and, halos included, it holds at
// most kLightDig digits and runs.  Lists in arbitrary order (the window counts
// and spans place the records canonically).
__global__ void __launch_bounds__(256) k_find_classify(DevGeom G, DevWork W, unsigned int n_windows) {
  const int lane = threadIdx.x & 31;
  for (unsigned long long b = (blockIdx.x * (unsigned long long)blockDim.x) + (threadIdx.x & ~31u); b < n_windows;
       b += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned w = (unsigned)b + lane;
    bool light = false;
    if (w < n_windows) {
      const int frs = window_frs(G, w);
      const int f = frs & 0xffff, r = (frs >> 16) & 0xff, s = (frs >> 24) & 0xff;
      PageHdr h, hp, hn;
      const uint64_t o = W.page_offsets[w];
      bool ok = parse_header(reinterpret_cast<const uint4*>(W.pages + (o <= W.pages_bytes ? o : 0)), o,
                             W.pages_bytes, h) && h.sector == s && h.row == r && h.frag == f;
      int nd = ok ? h.n_dig : 0, nr = ok ? h.n_runs : 0;
      if (ok && f > 0) {
        const uint64_t op = W.page_offsets[w - 1];
        ok = parse_header(reinterpret_cast<const uint4*>(W.pages + (op <= W.pages_bytes ? op : 0)), op,
                          W.pages_bytes, hp);
        nd += ok ? hp.n_dig - hp.hi_dig : 0;
        nr += ok ? hp.n_runs - hp.hi_runs : 0;
      }
      if (ok && f + 1 < G.n_frag) {
        const uint64_t on = W.page_offsets[w + 1];
        ok = parse_header(reinterpret_cast<const uint4*>(W.pages + (on <= W.pages_bytes ? on : 0)), on,
                          W.pages_bytes, hn);
        nd += ok ? hn.lo_dig : 0;
        nr += ok ? hn.lo_runs : 0;
      }
      light = ok && nd <= kLightDig && nr <= kLightDig;
    }
    const bool valid = w < n_windows;
    const uint32_t ml = __ballot_sync(0xffffffffu, valid && light), mh = __ballot_sync(0xffffffffu, valid && !light);
    unsigned long long bl = 0, bh = 0;
    if (lane == 0) {
      if (ml) bl = atomicAdd(&W.ctr[CTR_NLIGHT], (unsigned long long)__popc(ml));
      if (mh) bh = atomicAdd(&W.ctr[CTR_NHEAVY], (unsigned long long)__popc(mh));
    }
    bl = __shfl_sync(0xffffffffu, bl, 0);
    bh = __shfl_sync(0xffffffffu, bh, 0);
    const uint32_t lt = (1u << lane) - 1u;
    if (valid && light) W.light_list[bl + __popc(ml & lt)] = w;
    if (valid && !light) W.heavy_list[bh + __popc(mh & lt)] = w;
  }
}

// Warp inclusive scan.
__device__ __forceinline__ int warp_incl(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

__global__ void __launch_bounds__(kLightWarps * 32, kLightBlocksPerSm)
k_find_light(DevGeom G, DevParams P, DevWork W, unsigned int n_windows) {
  __shared__ LightWarp LS[kLightWarps];
  LightWarp& L = LS[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const unsigned long long n_light = W.ctr[CTR_NLIGHT];
  const int T = G.n_time_bins;
  // tickets one window ahead: the next window's page is prefetched into L2
  // while this one is processed
  unsigned t = 0;
  if (lane == 0) t = atomicAdd(&W.tickets[TK_LIGHT], 1u);
  t = __shfl_sync(0xffffffffu, t, 0);
  while (true) {
    if ((unsigned long long)t >= n_light) break;
    const unsigned w = W.light_list[t];
    unsigned tn = 0;
    if (lane == 0) {
      tn = atomicAdd(&W.tickets[TK_LIGHT], 1u);
      if ((unsigned long long)tn < n_light) {
        const unsigned wn = W.light_list[tn];   // its own page (the halos are a few bytes)
        const unsigned long long lo = W.page_offsets[wn];
        const unsigned long long hi = wn + 1 < n_windows ? W.page_offsets[wn + 1] : W.pages_bytes;
        if (lo < hi && lo < W.pages_bytes && (lo & 15) == 0)
          prefetch_l2(W.pages + lo, min(hi, (unsigned long long)W.pages_bytes) - lo);
      }
    }
    t = __shfl_sync(0xffffffffu, tn, 0);
    const int frs = window_frs(G, w);
    const int f = frs & 0xffff, r = (frs >> 16) & 0xff, s = (frs >> 24) & 0xff;
    const int np = G.npads[r];
    // ---- the three segments, staged in one round trip: the own page whole,
    // the neighbours' halo entries / runs / ADC words (headers valid: checked
    // by the classification)
    LightSeg sg[3];
    bool bad = false;
    {
      PageHdr h, hp, hn;
      const uint64_t o = W.page_offsets[w];
      const uint64_t op = f > 0 ? W.page_offsets[w - 1] : 0ull;
      const uint64_t on = f + 1 < G.n_frag ? W.page_offsets[w + 1] : 0ull;
      parse_header(reinterpret_cast<const uint4*>(W.pages + o), o, W.pages_bytes, h);
      if (f > 0) parse_header(reinterpret_cast<const uint4*>(W.pages + op), op, W.pages_bytes, hp);
      if (f + 1 < G.n_frag) parse_header(reinterpret_cast<const uint4*>(W.pages + on), on, W.pages_bytes, hn);
      if (h.len > (uint32_t)kLightOwn) bad = true;
      const uint8_t* own = reinterpret_cast<const uint8_t*>(L.own);
      const uint4* src = reinterpret_cast<const uint4*>(W.pages + o);
      for (int i = lane; i < (int)(min(h.len, (uint32_t)kLightOwn) / 16); i += 32) L.own[i] = __ldg(src + i);
      sg[1] = LightSeg{reinterpret_cast<const uint16_t*>(own + 32), reinterpret_cast<const uint16_t*>(own + 32 + 2 * h.n_tb),
                       reinterpret_cast<const uint32_t*>(own + h.body), h.n_tb, h.n_runs, h.n_dig, 0, kHalo, kFrag * f};
      sg[0] = LightSeg{nullptr, nullptr, nullptr, 0, 0, 0, 0, kHalo - kFrag, kFrag * (f - 1)};
      sg[2] = LightSeg{nullptr, nullptr, nullptr, 0, 0, 0, 0, kHalo + kFrag, kFrag * (f + 1)};
      uint16_t* hs0 = reinterpret_cast<uint16_t*>(L.halo[0]);
      uint16_t* hs1 = reinterpret_cast<uint16_t*>(L.halo[1]);
      if (f > 0) {
        const uint32_t e0 = 32 + 2 * hp.hi_tb, e1 = 32 + 2 * hp.n_tb;
        const uint32_t r0 = 32 + 2 * hp.n_tb + 2 * hp.hi_runs, r1 = 32 + 2 * hp.n_tb + 2 * hp.n_runs;
        const uint32_t a0 = hp.body + 4 * (hp.hi_dig / 3), a1 = hp.body + 4 * ((hp.n_dig + 2) / 3);
        if (e1 - e0 > 16 || r1 - r0 > 2 * kLightDig || a1 - a0 > kLightHalo - kHaloAdcAt) bad = true;
        if (!bad) {
          copy_u16_warp(hs0, W.pages + op, e0, e1);
          copy_u16_warp(hs0 + 8, W.pages + op, r0, r1);
          copy_u16_warp(hs0 + kHaloAdcAt / 2, W.pages + op, a0, a1);
        }
        sg[0].ent = hs0; sg[0].run = hs0 + 8; sg[0].adc = reinterpret_cast<const uint32_t*>(hs0 + kHaloAdcAt / 2);
        sg[0].ne = hp.n_tb - hp.hi_tb; sg[0].nrun = hp.n_runs - hp.hi_runs; sg[0].ndig = hp.n_dig - hp.hi_dig;
        sg[0].dfirst = hp.hi_dig % 3;
      }
      if (f + 1 < G.n_frag) {
        const uint32_t e1 = 32 + 2 * hn.lo_tb;
        const uint32_t r0 = 32 + 2 * hn.n_tb, r1 = r0 + 2 * hn.lo_runs;
        const uint32_t a0 = hn.body, a1 = hn.body + 4 * ((hn.lo_dig + 2) / 3);
        if (e1 - 32 > 16 || r1 - r0 > 2 * kLightDig || a1 - a0 > kLightHalo - kHaloAdcAt) bad = true;
        if (!bad) {
          copy_u16_warp(hs1, W.pages + on, 32, e1);
          copy_u16_warp(hs1 + 8, W.pages + on, r0, r1);
          copy_u16_warp(hs1 + kHaloAdcAt / 2, W.pages + on, a0, a1);
        }
        sg[2].ent = hs1; sg[2].run = hs1 + 8; sg[2].adc = reinterpret_cast<const uint32_t*>(hs1 + kHaloAdcAt / 2);
        sg[2].ne = hn.lo_tb; sg[2].nrun = hn.lo_runs; sg[2].ndig = hn.lo_dig;
      }
      bad = __any_sync(0xffffffffu, bad);
      __syncwarp();
    }
    const int ne = sg[0].ne + sg[1].ne + sg[2].ne;
    const int nrun = sg[0].nrun + sg[1].nrun + sg[2].nrun;
    const int ndig = sg[0].ndig + sg[1].ndig + sg[2].ndig;
    bad = bad || nrun > kLightDig || ndig > kLightDig;
    for (int i = lane; i < kWinT + 2; i += 32) { L.row0[i] = 0; L.row1[i] = 0; }
    // ---- entries: run counts -> each run's time bin
    {
      int carry = 0, cnt[3] = {0, 0, 0};
      for (int c0 = 0; c0 < ne && !bad; c0 += 32) {
        const int e = c0 + lane;
        int nr = 0, t_in = 0, k = 0;
        if (e < ne) {
          k = e < sg[0].ne ? 0 : (e < sg[0].ne + sg[1].ne ? 1 : 2);
          const int el = e - (k == 0 ? 0 : (k == 1 ? sg[0].ne : sg[0].ne + sg[1].ne));
          const LightSeg& g = sg[k];
          const uint32_t v = g.ent[el];
          t_in = (int)(v & 0xffu);
          nr = (int)(v >> 8);
          const int tt = t_in + g.tt_base;
          if (nr < 1 || tt < 0 || tt >= kWinT || g.t_base + t_in >= T) bad = true;
          if (el > 0 && (int)(g.ent[el - 1] & 0xffu) >= t_in) bad = true;
        }
        const int incl = warp_incl(nr);
        int r0 = carry + incl - nr;
        for (int q = 0; q < nr; q++)
          if (r0 + q < kLightDig) L.run_t[r0 + q] = (uint8_t)t_in;
#pragma unroll
        for (int kk = 0; kk < 3; kk++) cnt[kk] += __reduce_add_sync(0xffffffffu, (e < ne && k == kk) ? nr : 0);
        carry += __shfl_sync(0xffffffffu, incl, 31);
        bad = __any_sync(0xffffffffu, bad);
      }
      // every segment's entries list exactly its runs
      if (cnt[0] != sg[0].nrun || cnt[1] != sg[1].nrun || cnt[2] != sg[2].nrun) bad = true;
    }
    __syncwarp();
    // ---- runs: digit offsets -> each digit's pixel
    if (!bad) {
      int carry = 0, cnt[3] = {0, 0, 0};
      for (int c0 = 0; c0 < nrun && !bad; c0 += 32) {
        const int rr = c0 + lane;
        int len = 0, ps = 0, k = 0;
        if (rr < nrun) {
          k = rr < sg[0].nrun ? 0 : (rr < sg[0].nrun + sg[1].nrun ? 1 : 2);
          const int rl = rr - (k == 0 ? 0 : (k == 1 ? sg[0].nrun : sg[0].nrun + sg[1].nrun));
          const LightSeg& g = sg[k];
          const uint32_t rv = g.run[rl];
          ps = (int)(rv & 0xffu);
          len = (int)(rv >> 8);
          if (len < 1 || ps + len > np) bad = true;
          if (rl > 0 && L.run_t[rr - 1] == L.run_t[rr]) {   // same time bin: ascending, disjoint
            const uint32_t pv = g.run[rl - 1];
            if (ps < (int)(pv & 0xffu) + (int)(pv >> 8)) bad = true;
          }
        }
        const int incl = warp_incl(len);
        const int d0 = carry + incl - len;
        if (!bad && rr < nrun) {
          const int tt = (int)L.run_t[rr] + sg[k].tt_base;
          for (int q = 0; q < len; q++)
            if (d0 + q < kLightDig) {
              L.dt[d0 + q] = (uint16_t)tt;
              L.dp[d0 + q] = (uint8_t)(ps + q);
            }
        }
#pragma unroll
        for (int kk = 0; kk < 3; kk++) cnt[kk] += __reduce_add_sync(0xffffffffu, (rr < nrun && k == kk) ? len : 0);
        carry += __shfl_sync(0xffffffffu, incl, 31);
        bad = __any_sync(0xffffffffu, bad);
      }
      if (cnt[0] != sg[0].ndig || cnt[1] != sg[1].ndig || cnt[2] != sg[2].ndig) bad = true;
    }
    __syncwarp();
    // ---- digits: ADC values, row bounds (digits sorted by row, then pad:
    // segments in time order, entries ascending in time, runs of a time bin
    // ascending and disjoint, as checked above)
    if (!bad) {
      for (int d = lane; d < ndig; d += 32) {
        const int k = d < sg[0].ndig ? 0 : (d < sg[0].ndig + sg[1].ndig ? 1 : 2);
        const int dl = d - (k == 0 ? 0 : (k == 1 ? sg[0].ndig : sg[0].ndig + sg[1].ndig));
        const int idx = sg[k].dfirst + dl;
        const uint32_t word = sg[k].adc[idx / 3];
        L.dq[d] = (uint16_t)((word >> (10 * (idx % 3))) & 1023u);
        const int tt = L.dt[d];
        if (d == 0 || L.dt[d - 1] != tt) L.row0[tt] = (uint16_t)d;
        if (d == ndig - 1 || L.dt[d + 1] != tt) L.row1[tt] = (uint16_t)(d + 1);
      }
    }
    __syncwarp();
    if (bad) {
      if (lane == 0) {
        atomicOr(W.err, kErrCorrupt);
        W.win_cnt[w] = 0ull;
        W.win_soff[w] = 0u;
      }
      __syncwarp();
      continue;
    }
    // ---- step 2: peaks (rows 1..260), one digit a lane
    for (int c0 = 0; c0 < ndig; c0 += 32) {
      const int d = c0 + lane;
      bool pkf = false;
      if (d < ndig) {
        const int tt = L.dt[d], p = L.dp[d], q = L.dq[d];
        if (tt >= 1 && tt <= kWinT - 2 && q >= P.q_peak_min) {
          const int lo = max(max(light_q(L, tt - 1, p - 1, np), light_q(L, tt - 1, p, np)),
                             max(light_q(L, tt - 1, p + 1, np), light_q(L, tt, p - 1, np)));
          const int hi = max(max(light_q(L, tt, p + 1, np), light_q(L, tt + 1, p - 1, np)),
                             max(light_q(L, tt + 1, p, np), light_q(L, tt + 1, p + 1, np)));
          pkf = q > lo && q >= hi;
        }
      }
      const uint32_t m = __ballot_sync(0xffffffffu, pkf);
      if (lane == 0) L.pk[c0 >> 5] = m;
    }
    __syncwarp();
    // ---- step 2b (noise suppression, optional): an own peak with a greater
    // step-2 peak on its 5x5 ring and a shallow dip towards it is dropped
    for (int c0 = 0; c0 < ndig; c0 += 32) {
      const int d = c0 + lane;
      bool keep = d < ndig && ((L.pk[c0 >> 5] >> lane) & 1u);
      if (keep && P.ns_min_dip > 0 && L.dt[d] >= kHalo && L.dt[d] < kHalo + kFrag) {
        const int tt = L.dt[d], p = L.dp[d], qc = L.dq[d];
        for (int dtt = -2; dtt <= 2 && keep; dtt++)
          for (int dpp = -2; dpp <= 2 && keep; dpp++) {
            if (dtt > -2 && dtt < 2 && dpp > -2 && dpp < 2) continue;   // the ring only
            const int i = light_find(L, tt + dtt, p + dpp, np);
            if (i < 0 || !((L.pk[i >> 5] >> (i & 31)) & 1u)) continue;
            const int qn = L.dq[i];
            // greater key: more charge, or equal charge and a lower (t, p) index
            if (qn < qc || (qn == qc && (dtt > 0 || (dtt == 0 && dpp > 0)))) continue;
            const int it = dtt > 0 ? 1 : (dtt < 0 ? -1 : 0), ip = dpp > 0 ? 1 : (dpp < 0 ? -1 : 0);
            if (qc - light_q(L, tt + it, p + ip, np) < P.ns_min_dip) keep = false;
          }
      }
      const uint32_t m = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) L.sv[c0 >> 5] = m;
    }
    __syncwarp();
    // ---- steps 3-4: the own surviving peaks (rows 3..258) in canonical order
    int npk = 0;
    for (int c0 = 0; c0 < ndig; c0 += 32) {
      const int d = c0 + lane;
      const bool own = d < ndig && ((L.sv[c0 >> 5] >> lane) & 1u) && L.dt[d] >= kHalo && L.dt[d] < kHalo + kFrag;
      npk += __popc(__ballot_sync(0xffffffffu, own));
    }
    unsigned long long so = 0;
    if (lane == 0) {
      so = npk ? atomicAdd(&W.ctr[CTR_SCURSOR], (unsigned long long)npk) : 0ull;
      if (so + npk > W.cap_cl) atomicOr(W.err, kErrOverflowCl);
      W.win_cnt[w] = (unsigned long long)npk;
      W.win_soff[w] = (uint32_t)min(so, (unsigned long long)W.cap_cl);
    }
    so = __shfl_sync(0xffffffffu, so, 0);
    int rank0 = 0;
    for (int c0 = 0; c0 < ndig && npk; c0 += 32) {
      const int d = c0 + lane;
      const bool own = d < ndig && ((L.sv[c0 >> 5] >> lane) & 1u) && L.dt[d] >= kHalo && L.dt[d] < kHalo + kFrag;
      const uint32_t m = __ballot_sync(0xffffffffu, own);
      if (own) {
        const int tt = L.dt[d], p = L.dp[d];
        int q[5][5];
        bool other = false;
#pragma unroll
        for (int a = 0; a < 5; a++)
#pragma unroll
          for (int b = 0; b < 5; b++) {
            if (a == 2 && b == 2) { q[a][b] = L.dq[d]; continue; }
            const int i = light_find(L, tt + a - 2, p + b - 2, np);
            q[a][b] = i < 0 ? 0 : (int)L.dq[i];
            if (i >= 0 && ((L.pk[i >> 5] >> (i & 31)) & 1u)) other = true;
          }
        uint4 rec;
        int4 xyz;
        cluster_record(q, other, np, T, s, r, f, tt, p, G.xrow[r], rec, xyz);
        const unsigned long long idx = so + rank0 + __popc(m & ((1u << lane) - 1u));
        if (idx < W.cap_cl) reinterpret_cast<uint4*>(W.scratch_cl)[idx] = rec;
      }
      rank0 += __popc(m);
    }
    __syncwarp();
  }
}

// Places every unit's scratch span at its canonical offset (win_cnt holds the
// exclusive scan of the unit counts; the total is in ctr[CTR_NCL]) and derives
// the (X, Y, Z, t_peak) arrays and the row starts.  A unit is a window (upw =
// 1) or a time chunk of one (upw chunks per window, in time order).  One warp
// per unit.
__global__ void __launch_bounds__(256)
k_compact_clusters(DevGeom G, DevWork W, unsigned int n_windows, int upw) {
  const int lane = threadIdx.x & 31;
  const unsigned long long total = W.ctr[CTR_NCL];
  const unsigned long long cap = W.cap_cl;
  const unsigned long long per_row = (unsigned long long)G.n_frag * upw;   // units per (sector, row)
  for (unsigned long long w = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5; w < n_windows;
       w += ((unsigned long long)gridDim.x * blockDim.x) >> 5) {
    const unsigned long long b = W.win_cnt[w];
    const unsigned long long e = (w + 1 < n_windows) ? W.win_cnt[w + 1] : total;
    const unsigned long long so = W.win_soff[w];
    if (lane == 0 && w % per_row == 0) W.row_start[w / per_row] = (uint32_t)min(b, cap);
    if (lane == 0 && w == n_windows - 1) W.row_start[G.n_sectors * G.n_rows] = (uint32_t)min(total, cap);
    for (unsigned long long k = lane; b + k < e; k += 32) {
      if (b + k >= cap || so + k >= cap) break;
      const uint4 rec = __ldg(reinterpret_cast<const uint4*>(W.scratch_cl) + so + k);
      const unsigned long long idx = b + k;
      reinterpret_cast<uint4*>(W.clusters)[idx] = rec;
      const int r = (rec.z >> 24) & 0xff;
      const int pad_fp = rec.x & 0xffff, time_fp = rec.x >> 16, t = rec.w & 0xffff;
      const int rr = r < G.n_rows ? r : 0;
      W.cl_x[idx] = G.xrow[rr];
      W.cl_y[idx] = 2 * (pad_fp - 128 * (G.npads[rr] - 1));
      W.cl_z[idx] = 5 * (32768 * (t / kFrag) + time_fp - 512);
      W.cl_t[idx] = t;
    }
  }
}

size_t find_smem_bytes(int npmax, int nw) {
  size_t o = ((size_t)kWinT * (npmax + 2 * kPad) * 2 + 15) & ~(size_t)15;
  o += 2 * (size_t)kWinT * nw * 4 + (size_t)kRunMapWords * 4;
  o = (o + 15) & ~(size_t)15;
  o += 2 * kStage * 16 + 2 * kHaloStage + 4 * 16 + 4 * 8 + 34 * 8 + 16 * 4;
  o += (3 * sizeof(PageHdr) + 15) & ~(size_t)15;
  o += kList * 2 + kStage * 2 + ((size_t)kFrag * nw + 1) * 2 + 16;
  o += kMaxRuns;
  return o;
}

cudaError_t launch_scan(uint64_t* v, const unsigned long long* n_ptr, unsigned long long cap,
                        unsigned long long* state, unsigned int* ticket, unsigned long long* total, uint32_t* err,
                        int n_sm, cudaStream_t st);

// Raise the finder's dynamic shared-memory limit on the current device (once
// per context, outside any stream capture).
template <int kMode, bool kNs>
static cudaError_t prepare_mode() {
  cudaError_t e = cudaFuncSetAttribute(k_find_clusters<true, 256, kMode, kNs>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_find_clusters<true, 384, kMode, kNs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_find_clusters<true, 512, kMode, kNs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
  return e;
}

cudaError_t prepare_find() {
  cudaError_t e = prepare_mode<0, false>();
  if (e == cudaSuccess) e = prepare_mode<0, true>();
  if (e == cudaSuccess) e = prepare_mode<1, false>();
  if (e == cudaSuccess) e = prepare_mode<2, false>();
  if (e == cudaSuccess) e = prepare_mode<2, true>();
  return e;
}

cudaError_t launch_compact(const DevGeom& G, const DevWork& W, unsigned int n_units, int units_per_window, int n_sm,
                           cudaStream_t st);

template <int kMode, bool kNs>
static void launch_find_mode(const DevGeom& G, const DevParams& P, const DevWork& W, unsigned int n_windows,
                             unsigned grid, int threads, size_t sm, cudaStream_t st) {
  if (threads == 256)
    k_find_clusters<true, 256, kMode, kNs><<<grid, 256, sm, st>>>(G, P, W, n_windows);
  else if (threads == 512)
    k_find_clusters<true, 512, kMode, kNs><<<grid, 512, sm, st>>>(G, P, W, n_windows);
  else
    k_find_clusters<true, 384, kMode, kNs><<<grid, 384, sm, st>>>(G, P, W, n_windows);
}

cudaError_t launch_find(const DevGeom& G, const DevParams& P, const DevWork& W, unsigned int n_windows,
                        int n_sm, const LaunchCfg& L, cudaStream_t st, cudaStream_t aux, cudaEvent_t ev_fork,
                        cudaEvent_t ev_join, unsigned long long* win_scan_state, int* launches) {
  const size_t sm = find_smem_bytes(G.npmax, G.nw);
  // persistent CTAs: find_ctas_per_sm per SM (at most 2 fit the shared memory)
  unsigned int grid = (unsigned int)min((long long)n_windows, (long long)n_sm * L.find_ctas_per_sm);
  if (grid == 0) grid = 1;
  // step 2b (noise suppression) compiled in only where it is switched on
  const bool ns = P.ns_min_dip > 0;
  // light windows to one warp each (the fused finder, with or without step 2b),
  // on timeframes large enough that the light kernel's per-window latency
  // hides behind the block finder (a single sector gets slower with it)
  const bool light = W.light_list && W.heavy_list && !W.dense && n_windows >= kLightMinWindows;
  DevWork Wh = W;
  if (!light) Wh.light_list = Wh.heavy_list = nullptr;
  if (light) {
    // the light windows on a second stream, beside the block finder: whichever
    // kernel's blocks retire first leaves its SMs to the other
    unsigned gc = (unsigned)min((n_windows + 255ull) / 256ull, (unsigned long long)n_sm * 8);
    k_find_classify<<<gc ? gc : 1, 256, 0, st>>>(G, W, n_windows);
    cudaError_t e0 = cudaEventRecord(ev_fork, st);
    if (e0 == cudaSuccess) e0 = cudaStreamWaitEvent(aux, ev_fork, 0);
    if (e0 != cudaSuccess) return e0;
    k_find_light<<<(unsigned)(n_sm * kLightBlocksPerSm), kLightWarps * 32, 0, aux>>>(G, P, W, n_windows);
    e0 = cudaEventRecord(ev_join, aux);
    if (e0 != cudaSuccess) return e0;
    *launches += 2;
  }
  if (W.dense) {
    // dense-plane variant: decode every window into the plane, then find
    launch_find_mode<1, false>(G, P, Wh, n_windows, grid, L.find_threads, sm, st);
    if (ns) launch_find_mode<2, true>(G, P, Wh, n_windows, grid, L.find_threads, sm, st);
    else launch_find_mode<2, false>(G, P, Wh, n_windows, grid, L.find_threads, sm, st);
    *launches += 1;
  } else if (ns) {
    launch_find_mode<0, true>(G, P, Wh, n_windows, grid, L.find_threads, sm, st);
  } else {
    launch_find_mode<0, false>(G, P, Wh, n_windows, grid, L.find_threads, sm, st);
  }
  if (light) {
    const cudaError_t e1 = cudaStreamWaitEvent(st, ev_join, 0);
    if (e1 != cudaSuccess) return e1;
  }
  cudaError_t e = launch_scan(reinterpret_cast<uint64_t*>(W.win_cnt), W.ctr + CTR_NWIN, n_windows, win_scan_state,
                              W.tickets + TK_SCAN_W, W.ctr + CTR_NCL, W.err, n_sm, st);
  if (e != cudaSuccess) return e;
  e = launch_compact(G, W, n_windows, 1, n_sm, st);
  *launches += 3;
  return e;
}

cudaError_t launch_compact(const DevGeom& G, const DevWork& W, unsigned int n_units, int units_per_window, int n_sm,
                           cudaStream_t st) {
  unsigned long long gc = ((unsigned long long)n_units * 32 + 255) / 256;
  if (gc > (unsigned long long)n_sm * 8) gc = (unsigned long long)n_sm * 8;
  k_compact_clusters<<<(unsigned)(gc ? gc : 1), 256, 0, st>>>(G, W, n_units, units_per_window);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the finder.  The look-back states and the control
// words (counters, error word, ticket) live in this file-scope array instead
// of memory from cudaMalloc; every GPU that loads the library holds it until
// the process exits.
constexpr unsigned kNoAllocMaxWindows = 65536;
constexpr unsigned kNoAllocCtrlWords = 32;   // CTR_COUNT counters + error word + tickets
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocMaxWindows + kNoAllocCtrlWords];

namespace {
std::mutex g_noalloc_mu;
unsigned long long* g_noalloc_addr[64];      // device address of the array, per device
bool g_noalloc_ready[64];
}  // namespace

}  // namespace tpc

extern "C" tpc_status tpc_find_clusters_noalloc(const tpc_geometry* geom, const tpc_params* params, int device,
                                                const void* pages, uint64_t pages_bytes,
                                                const uint64_t* page_offsets, uint32_t n_time_bins,
                                                tpc_cluster* clusters, uint64_t cap, uint64_t* n_clusters,
                                                void* stream) {
  using namespace tpc;
  auto fail = [](tpc_status st, const char* msg) { set_last_error(msg); return st; };
  if (!geom || !pages || !page_offsets || !clusters || !n_clusters)
    return fail(TPC_E_INVAL, "tpc_find_clusters_noalloc: null argument");
  if (((uintptr_t)pages & 15) || ((uintptr_t)clusters & 15))
    return fail(TPC_E_INVAL, "tpc_find_clusters_noalloc: pages and clusters must be 16-byte aligned");
  if (n_time_bins < 1 || n_time_bins > 65535 || pages_bytes < 32)
    return fail(TPC_E_INVAL, "tpc_find_clusters_noalloc: n_time_bins or pages_bytes out of range");
  const int q_peak_min = params ? params->q_peak_min : 10;
  if (params && params->version != TPC_PARAMS_VERSION)
    return fail(TPC_E_INVAL, "tpc_find_clusters_noalloc: params version mismatch");
  if (q_peak_min < 1 || q_peak_min > 1023) return fail(TPC_E_INVAL, "tpc_find_clusters_noalloc: bad q_peak_min");
  const int ns_min_dip = params ? params->ns_min_dip : 0;
  if (ns_min_dip < 0 || ns_min_dip > 1023) return fail(TPC_E_INVAL, "tpc_find_clusters_noalloc: bad ns_min_dip");
  if (params && params->split_charge)
    return fail(TPC_E_INVAL, "tpc_find_clusters_noalloc: split_charge is not supported here");
  const unsigned long long nfrag = (n_time_bins + kFrag - 1) / kFrag;
  const unsigned long long nwin = (unsigned long long)geom->n_sectors * geom->n_rows * nfrag;
  if (nwin > kNoAllocMaxWindows)
    return fail(TPC_E_INVAL,
                "tpc_find_clusters_noalloc: the timeframe has more windows (sector x row x 256-bin fragment) "
                "than the 65536 its fixed scratch holds");
  if (device < 0 || device >= 64) return fail(TPC_E_INVAL, "tpc_find_clusters_noalloc: bad device");
  int prev_dev = -1;
  if (cudaGetDevice(&prev_dev) != cudaSuccess) return fail(TPC_E_CUDA, "cudaGetDevice failed");
  if (prev_dev != device && cudaSetDevice(device) != cudaSuccess) return fail(TPC_E_CUDA, "cudaSetDevice failed");
  struct Restore {
    int d, p;
    ~Restore() { if (p >= 0 && p != d) cudaSetDevice(p); }
  } restore{device, prev_dev};
  // one-time set-up on this device (with the device current): the array's
  // device address and the kernel's shared-memory limit
  const size_t smem = find_smem_bytes(geom->npmax, (geom->npmax + 31) / 32);
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ready[device]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
        return fail(TPC_E_CUDA, "tpc_find_clusters_noalloc: cudaGetSymbolAddress failed");
      if (cudaFuncSetAttribute(k_find_clusters<false, kFindThreads, 0, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess ||
          cudaFuncSetAttribute(k_find_clusters<false, kFindThreads, 0, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess)
        return fail(TPC_E_CUDA, "tpc_find_clusters_noalloc: cudaFuncSetAttribute failed");
      g_noalloc_addr[device] = static_cast<unsigned long long*>(ptr);
      g_noalloc_ready[device] = true;
    }
  }
  if (smem > 227 * 1024) return fail(TPC_E_INVAL, "tpc_find_clusters_noalloc: rows too wide");
  unsigned long long* scratch = g_noalloc_addr[device];
  DevGeom G{};
  G.n_sectors = geom->n_sectors;
  G.n_phys = geom->n_sectors;
  G.n_events = 1;
  G.n_rows = geom->n_rows;
  G.npmax = geom->npmax;
  G.nw = (geom->npmax + 31) / 32;
  G.n_time_bins = (int)n_time_bins;
  G.n_frag = (int)nfrag;
  for (int r = 0; r < geom->n_rows; r++) { G.npads[r] = geom->npads[r]; G.xrow[r] = 64 * geom->row_x[r]; }
  DevParams P{};
  P.q_peak_min = q_peak_min;
  P.ns_min_dip = ns_min_dip;
  DevWork W{};
  W.pages = static_cast<const uint8_t*>(pages);
  W.page_offsets = page_offsets;
  W.pages_bytes = pages_bytes;
  W.clusters = clusters;
  W.cap_cl = cap;
  W.win_state = scratch;
  W.ctr = scratch + kNoAllocMaxWindows;
  W.err = reinterpret_cast<uint32_t*>(W.ctr + CTR_COUNT);
  W.tickets = reinterpret_cast<unsigned int*>(W.ctr + CTR_COUNT + 1);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: clear what must start at zero
  if (cudaMemsetAsync(W.ctr, 0, kNoAllocCtrlWords * 8, st) != cudaSuccess ||
      cudaMemsetAsync(W.win_state, 0, nwin * 8, st) != cudaSuccess)
    return fail(TPC_E_CUDA, "tpc_find_clusters_noalloc: cudaMemsetAsync failed");
  int n_sm = 148;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
  unsigned grid = (unsigned)std::min<unsigned long long>(nwin, (unsigned long long)n_sm * 2);
  if (ns_min_dip > 0)
    k_find_clusters<false, kFindThreads, 0, true><<<grid ? grid : 1, kFindThreads, smem, st>>>(G, P, W, (unsigned)nwin);
  else
    k_find_clusters<false, kFindThreads, 0, false><<<grid ? grid : 1, kFindThreads, smem, st>>>(G, P, W, (unsigned)nwin);
  if (cudaGetLastError() != cudaSuccess) return fail(TPC_E_CUDA, "tpc_find_clusters_noalloc: launch failed");
  unsigned long long ctrl[CTR_COUNT + 1];
  if (cudaMemcpyAsync(ctrl, W.ctr, sizeof ctrl, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(TPC_E_CUDA, "tpc_find_clusters_noalloc: device error");
  const uint32_t err = static_cast<uint32_t>(ctrl[CTR_COUNT] & 0xffffffffu);
  *n_clusters = ctrl[CTR_NCL];
  if (err & kErrCorrupt) return fail(TPC_E_CORRUPT, "tpc_find_clusters_noalloc: corrupt ZS page");
  if (err & kErrTimeout) return fail(TPC_E_TIMEOUT, "tpc_find_clusters_noalloc: look-back wait gave up");
  if (err & kErrOverflowCl) return fail(TPC_E_OVERFLOW, "tpc_find_clusters_noalloc: more clusters than cap");
  if (err) return fail(TPC_E_DEVICE, "tpc_find_clusters_noalloc: device error word set");
  return TPC_OK;
}

