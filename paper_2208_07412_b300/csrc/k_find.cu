// k_find.cu — ZS decode + 3x3 peak finder + 5x5 cluster moments + stable
// compaction, fused in one persistent kernel (steps 1-4 of the library's
// definition; the paper's section "Hardware and data flow" places this first
// step of the TPC reconstruction on the EPN GPUs, after FPGA zero suppression).
//
// One CTA iteration processes one window = (sector, row, 256-bin fragment).
// Memory round trips are the cost to avoid: the next window's ticket is taken
// a window ahead, the page is staged in shared memory by one coalesced copy
// (issued together with the neighbours' headers), and the neighbours' 3-bin
// halo byte ranges by a second one; everything after that reads shared memory.
// Digits are decoded into a plane guarded by an occupancy bitmap: only the
// bitmap (5 KB) is cleared, never the 72 KB plane, so the work scales with the
// digits, not with the pixels.  Digits, then peaks, are ranked by popcount
// prefixes over the bitmap words, which follow the canonical (t, pad) order,
// so every thread gets an equal share of the peak tests and of the clusters.
// A decoupled look-back over the windows (handed out in index order by the
// ticket) gives each window's global offset; its aggregate is published before
// the clusters are built, so the wait overlaps that work, and the clusters are
// written once, coalesced, at their final place.
#include "tpc_internal.cuh"

namespace tpc {

constexpr int kFindThreads = 256;

struct PageHdr {
  uint32_t len;
  int n_tb, n_runs, n_dig, sector, row, frag, magic;
  int lo_tb, lo_runs, lo_dig, hi_tb, hi_runs, hi_dig;
  uint32_t body;   // byte offset of the ADC words
};

// Parse and validate a 32-byte page header (from shared or global memory) of
// the page at byte offset `off` of a `pages_bytes` buffer.
__device__ __forceinline__ bool parse_header(const uint4* p, uint64_t off, uint64_t pages_bytes, PageHdr& h) {
  if ((off & 15) || off + 32 > pages_bytes) return false;
  const uint4 a = p[0], b = p[1];
  h.len = a.x;
  h.n_tb = a.y & 0xffff; h.n_runs = a.y >> 16;
  h.n_dig = a.z & 0xffff; h.sector = (a.z >> 16) & 0xff; h.row = a.z >> 24;
  h.frag = a.w & 0xffff; h.magic = a.w >> 16;
  h.lo_tb = b.x & 0xffff; h.lo_runs = b.x >> 16; h.lo_dig = b.y & 0xffff;
  h.hi_tb = b.y >> 16; h.hi_runs = b.z & 0xffff; h.hi_dig = b.z >> 16;
  const uint64_t body = (32ull + 2ull * h.n_tb + 2ull * h.n_runs + 3ull) & ~3ull;
  h.body = (uint32_t)body;
  if (h.magic != (int)TPC_ZS_MAGIC || (h.len & 15) || off + h.len > pages_bytes ||
      body + 4ull * ((h.n_dig + 2) / 3) > h.len)
    return false;
  if (h.n_tb > kFrag || h.lo_tb > h.n_tb || h.hi_tb > h.n_tb || h.lo_runs > h.n_runs ||
      h.hi_runs > h.n_runs || h.lo_dig > h.n_dig || h.hi_dig > h.n_dig)
    return false;
  return true;
}

constexpr int kStage = 256;                  // clusters staged in shared memory before the look-back
constexpr int kOwnStage = 2 * kStage * 16;   // bytes; the page is staged in the same buffer first
constexpr int kHaloStage = 2048;             // bytes per neighbouring page's halo ranges
constexpr int kHaloRunOff = 16, kHaloAdcOff = 800;

struct FindSmem {
  uint16_t* plane;     // [kWinT][npmax]
  uint32_t* occ;       // [kWinT][nw]
  uint32_t* pk;        // [kWinT][nw]
  uint16_t* wpre;      // digit rank prefix over the words of plane rows 1..260
  uint16_t* ppre;      // own-peak rank prefix over the words of rows 3..258
  uint4* st_rec;       // [kStage] staged cluster records (first: the staged page)
  int4* st_xyz;        // [kStage] staged (X, Y, Z, t_peak)
  uint8_t* halo;       // [2][kHaloStage] halo ranges of the previous / next page
  uint4* hdr;          // [4] headers of the previous (0,1) and next (2,3) page
  unsigned long long* offs;  // [4] page offsets of windows w-1 .. w+2
  uint8_t* ent_t;      // [256]
  int32_t* ent_rs;     // [257]
  unsigned long long* scan;  // [34]
  int32_t* misc;       // [16]
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
// field (dfirst + k) % 3 of word (dfirst + k) / 3.  Pointers may address shared
// or global memory.
struct Seg {
  const uint16_t* ent; int ne;
  const uint16_t* run; int nrun;
  const uint32_t* adc; int dfirst; int ndig;
  int tt_base, t_base_abs;
  bool strict;                    // the window's own page: ordering and exact counts
};

// Decode a segment into plane rows tt = t_in + tt_base.  All reads are bounds-
// checked against the segment's counts and all writes against the plane.
// Returns true (block-uniform) if every check passed.
__device__ bool decode_seg(const Seg& g, int np, int stride, int nw, int T, const FindSmem& S) {
  const int tid = threadIdx.x;
  const int ne = g.ne;
  bool bad = ne < 0 || ne > kFrag;
  int t_in = 0, nr = 0;
  if (!bad && tid < ne) {
    const uint32_t v = g.ent[tid];
    t_in = v & 0xff;
    nr = v >> 8;
    const int tt = t_in + g.tt_base;
    if (nr < 1 || tt < 0 || tt >= kWinT || g.t_base_abs + t_in >= T) bad = true;
    if (g.strict && tid > 0 && (int)(g.ent[tid - 1] & 0xff) >= t_in) bad = true;
  }
  unsigned long long tot;
  const unsigned long long rs = block_excl_scan((unsigned long long)nr, S.scan, &tot);
  if (tid < ne) { S.ent_t[tid] = (uint8_t)t_in; S.ent_rs[tid] = (int32_t)rs; }
  const int nrun = (int)tot;
  if (nrun > g.nrun) bad = true;
  __syncthreads();
  unsigned long long dcarry = 0;
  for (int base = 0; base < nrun; base += blockDim.x) {
    const int j = base + tid;
    int ps = 0, len = 0, tt = 0;
    bool mine = j < nrun && j < g.nrun;
    if (mine) {
      const uint32_t v = g.run[j];
      ps = v & 0xff;
      len = v >> 8;
      int lo = 0, hi = ne - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.ent_rs[mid] <= j) lo = mid; else hi = mid - 1;
      }
      tt = (int)S.ent_t[lo] + g.tt_base;
      if (len < 1 || ps + len > np || tt < 0 || tt >= kWinT) { bad = true; mine = false; len = 0; }
      if (g.strict && j > S.ent_rs[lo]) {
        const uint32_t pv = g.run[j - 1];
        if ((int)ps < (int)(pv & 0xff) + (int)(pv >> 8)) bad = true;
      }
    }
    unsigned long long ctot;
    const unsigned long long doff = block_excl_scan((unsigned long long)len, S.scan, &ctot);
    const long long di = (long long)dcarry + (long long)doff;
    if (mine && di + len > g.ndig) { bad = true; mine = false; }
    if (mine) {
      uint16_t* prow = S.plane + tt * stride;
      for (int k = 0; k < len; k++) {
        const int d = g.dfirst + (int)di + k;
        prow[ps + k] = (uint16_t)((g.adc[d / 3] >> (10 * (d % 3))) & 1023u);
      }
      // occupancy bits for pads [ps, ps + len)
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
    dcarry += ctot;
  }
  if (g.strict && (nrun != g.nrun || (long long)dcarry != g.ndig)) bad = true;
  return !__syncthreads_or(bad);
}

// Copy the byte range [a, b) of a page (2-byte aligned, both in bounds) to dst
// as 16-bit words.
__device__ __forceinline__ void copy_u16(uint16_t* dst, const uint8_t* pg, uint32_t a, uint32_t b) {
  const uint16_t* src = reinterpret_cast<const uint16_t*>(pg + a);
  for (uint32_t i = threadIdx.x; i < (b - a) / 2; i += blockDim.x) dst[i] = __ldg(src + i);
}

__device__ __forceinline__ int qat(const FindSmem& S, int stride, int nw, int np, int tt, int p) {
  if (p < 0 || p >= np) return 0;
  return ((S.occ[tt * nw + (p >> 5)] >> (p & 31)) & 1u) ? (int)S.plane[tt * stride + p] : 0;
}
__device__ __forceinline__ bool pkat(const FindSmem& S, int nw, int np, int tt, int p) {
  if (p < 0 || p >= np) return false;
  return (S.pk[tt * nw + (p >> 5)] >> (p & 31)) & 1u;
}

__device__ __forceinline__ bool peak_test(const FindSmem& S, int stride, int nw, int np, int tt, int p, int q) {
  // neighbours with a lower linear index must be strictly lower in charge,
  // those with a higher index lower or equal: key = (q, -(t * npads + p))
  return q > qat(S, stride, nw, np, tt - 1, p - 1) && q > qat(S, stride, nw, np, tt - 1, p) &&
         q > qat(S, stride, nw, np, tt - 1, p + 1) && q > qat(S, stride, nw, np, tt, p - 1) &&
         q >= qat(S, stride, nw, np, tt, p + 1) && q >= qat(S, stride, nw, np, tt + 1, p - 1) &&
         q >= qat(S, stride, nw, np, tt + 1, p) && q >= qat(S, stride, nw, np, tt + 1, p + 1);
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

// Cluster of the peak at (tt, p): 5x5 window with the inner/outer rule.
__device__ __forceinline__ void make_cluster(const FindSmem& S, int stride, int nw, int np, int T, int s, int r,
                                             int f, int tt, int p, int xrow, uint4& rec, int4& xyz) {
  int Q = 0, Sp = 0, St = 0, Spp = 0, Stt = 0;
  bool excl = false, other = false;
#pragma unroll
  for (int dt = -2; dt <= 2; dt++) {
#pragma unroll
    for (int dp = -2; dp <= 2; dp++) {
      const int q = qat(S, stride, nw, np, tt + dt, p + dp);
      bool inc;
      if (dp >= -1 && dp <= 1 && dt >= -1 && dt <= 1) {
        inc = true;
      } else {
        const int ip = dp > 0 ? 1 : (dp < 0 ? -1 : 0), it = dt > 0 ? 1 : (dt < 0 ? -1 : 0);
        const int qi = qat(S, stride, nw, np, tt + it, p + ip);
        inc = qi > 0 && q <= qi;
        if (!inc && q > 0) excl = true;
      }
      if (inc) {
        Q += q; Sp += q * dp; St += q * dt; Spp += q * dp * dp; Stt += q * dt * dt;
      }
      if ((dp || dt) && pkat(S, nw, np, tt + dt, p + dp)) other = true;
    }
  }
  const int t_in = tt - kHalo;
  const int t = kFrag * f + t_in;
  const long long QQ = Q;
  const int pad_fp = 256 * p + (int)round_half_up(256LL * Sp, QQ);
  const int time_fp = 128 * (t_in + 4) + (int)round_half_up(128LL * St, QQ);
  const long long vp = round_half_up(16LL * ((long long)Spp * QQ - (long long)Sp * Sp), QQ * QQ);
  const long long vt = round_half_up(16LL * ((long long)Stt * QQ - (long long)St * St), QQ * QQ);
  const int flags = ((p == 0 || p == np - 1 || t == 0 || t == T - 1) ? TPC_CL_EDGE : 0) |
                    (excl ? TPC_CL_EXCLUDED : 0) | (other ? TPC_CL_NEIGHBOUR : 0);
  rec.x = (uint32_t)(pad_fp & 0xffff) | ((uint32_t)(time_fp & 0xffff) << 16);
  rec.y = (uint32_t)S.plane[tt * stride + p] | ((uint32_t)min(Q, 65535) << 16);
  rec.z = (uint32_t)min(vp, 255LL) | ((uint32_t)min(vt, 255LL) << 8) | ((uint32_t)flags << 16) |
          ((uint32_t)r << 24);
  rec.w = (uint32_t)t | ((uint32_t)p << 16) | ((uint32_t)s << 24);
  xyz = make_int4(xrow, 2 * (pad_fp - 128 * (np - 1)), 5 * (32768 * f + time_fp - 512), t);
}

__global__ void __launch_bounds__(kFindThreads, 2)
k_find_clusters(DevGeom G, DevParams P, DevWork W, unsigned int n_windows) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int stride = G.npmax, nw = G.nw;
  const int nrow_words = (kWinT - 2) * nw;   // plane rows 1 .. 260
  const int nown_words = kFrag * nw;         // plane rows 3 .. 258
  FindSmem S;
  {
    size_t o = 0;
    S.plane = reinterpret_cast<uint16_t*>(smem_raw + o);
    o += ((size_t)kWinT * stride * 2 + 15) & ~(size_t)15;
    S.occ = reinterpret_cast<uint32_t*>(smem_raw + o);
    o += (size_t)kWinT * nw * 4;
    S.pk = reinterpret_cast<uint32_t*>(smem_raw + o);
    o += (size_t)kWinT * nw * 4;
    o = (o + 15) & ~(size_t)15;
    S.st_rec = reinterpret_cast<uint4*>(smem_raw + o);
    o += kStage * 16;
    S.st_xyz = reinterpret_cast<int4*>(smem_raw + o);
    o += kStage * 16;
    S.halo = smem_raw + o;
    o += 2 * kHaloStage;
    S.hdr = reinterpret_cast<uint4*>(smem_raw + o);
    o += 4 * 16;
    S.offs = reinterpret_cast<unsigned long long*>(smem_raw + o);
    o += 4 * 8;
    S.scan = reinterpret_cast<unsigned long long*>(smem_raw + o);
    o += 34 * 8;
    S.ent_rs = reinterpret_cast<int32_t*>(smem_raw + o);
    o += 260 * 4;
    S.misc = reinterpret_cast<int32_t*>(smem_raw + o);
    o += 16 * 4;
    S.wpre = reinterpret_cast<uint16_t*>(smem_raw + o);
    o += ((size_t)nrow_words + 1) * 2;
    S.ppre = reinterpret_cast<uint16_t*>(smem_raw + o);
    o += ((size_t)nown_words + 1) * 2;
    S.ent_t = reinterpret_cast<uint8_t*>(smem_raw + o);
  }
  const int tid = threadIdx.x;
  const int wpt = (nrow_words + blockDim.x - 1) / blockDim.x;
  const int opt = (nown_words + blockDim.x - 1) / blockDim.x;
  uint8_t* own_stage = reinterpret_cast<uint8_t*>(S.st_rec);

  if (tid == 0) S.misc[1] = (int)atomicAdd(&W.tickets[TK_FIND], 1u);
  while (true) {
    // ---- 0. window w; take the next ticket now, one window ahead
    __syncthreads();
    const unsigned int w = (unsigned int)S.misc[1];
    if (w >= n_windows) break;
    if (tid < 4) {
      const long long j = (long long)w - 1 + tid;
      S.offs[tid] = (j >= 0 && j < (long long)n_windows) ? W.page_offsets[j] : ~0ull;
    }
    for (int i = tid; i < kWinT * nw; i += blockDim.x) S.occ[i] = 0u;
    __syncthreads();
    // every thread has read w: the slot may now receive the next ticket
    if (tid == 0) S.misc[1] = (int)atomicAdd(&W.tickets[TK_FIND], 1u);
    const int f = (int)(w % G.n_frag);
    const int sr = (int)(w / G.n_frag);
    const int r = sr % G.n_rows, s = sr / G.n_rows;
    const int np = G.npads[r];
    const int T = G.n_time_bins;
    const uint64_t off = S.offs[1];

    // ---- 1. one round trip: stage the page (length guessed from the next
    // page's offset) and load both neighbours' headers
    uint32_t copied = 0;
    if (off + 32 <= W.pages_bytes && (off & 15) == 0) {
      uint64_t guess = (S.offs[2] != ~0ull && S.offs[2] > off) ? S.offs[2] - off : W.pages_bytes - off;
      guess = min(guess, (uint64_t)kOwnStage);
      guess = min(guess, W.pages_bytes - off);
      copied = (uint32_t)(guess & ~15ull);
      const uint4* src = reinterpret_cast<const uint4*>(W.pages + off);
      for (uint32_t i = tid; i < copied / 16; i += blockDim.x) reinterpret_cast<uint4*>(own_stage)[i] = __ldg(src + i);
    }
    if (tid < 4) {
      const uint64_t o2 = S.offs[tid < 2 ? 0 : 2];
      const bool want = (tid < 2 ? f > 0 : f + 1 < G.n_frag) && o2 != ~0ull && (o2 & 15) == 0 && o2 + 32 <= W.pages_bytes;
      S.hdr[tid] = want ? __ldg(reinterpret_cast<const uint4*>(W.pages + o2) + (tid & 1)) : make_uint4(0, 0, 0, 0);
    }
    __syncthreads();

    // ---- 2. own header; neighbours' halo byte ranges in a second round trip
    PageHdr h, hp, hn;
    const uint8_t* own = copied >= 32 ? own_stage : W.pages + off;
    bool ok = parse_header(reinterpret_cast<const uint4*>(own), off, W.pages_bytes, h) && h.sector == s &&
              h.row == r && h.frag == f;
    const bool own_in_smem = ok && h.len <= copied;
    if (ok && !own_in_smem) own = W.pages + off;   // page larger than the stage: decode from global
    const bool okp = f > 0 && parse_header(S.hdr, S.offs[0], W.pages_bytes, hp) &&
                     2 * (hp.n_tb - hp.hi_tb) <= kHaloRunOff && 2 * (hp.n_runs - hp.hi_runs) <= kHaloAdcOff - kHaloRunOff &&
                     4 * ((hp.n_dig + 2) / 3 - hp.hi_dig / 3) <= kHaloStage - kHaloAdcOff;
    const bool okn = f + 1 < G.n_frag && parse_header(S.hdr + 2, S.offs[2], W.pages_bytes, hn) &&
                     2 * hn.lo_tb <= kHaloRunOff && 2 * hn.lo_runs <= kHaloAdcOff - kHaloRunOff &&
                     4 * ((hn.lo_dig + 2) / 3) <= kHaloStage - kHaloAdcOff;
    uint8_t* hprev = S.halo;
    uint8_t* hnext = S.halo + kHaloStage;
    if (okp) {
      const uint8_t* pg = W.pages + S.offs[0];
      copy_u16(reinterpret_cast<uint16_t*>(hprev), pg, 32 + 2 * hp.hi_tb, 32 + 2 * hp.n_tb);
      copy_u16(reinterpret_cast<uint16_t*>(hprev + kHaloRunOff), pg, 32 + 2 * hp.n_tb + 2 * hp.hi_runs,
               32 + 2 * hp.n_tb + 2 * hp.n_runs);
      copy_u16(reinterpret_cast<uint16_t*>(hprev + kHaloAdcOff), pg, hp.body + 4 * (hp.hi_dig / 3),
               hp.body + 4 * ((hp.n_dig + 2) / 3));
    }
    if (okn) {
      const uint8_t* pg = W.pages + S.offs[2];
      copy_u16(reinterpret_cast<uint16_t*>(hnext), pg, 32, 32 + 2 * hn.lo_tb);
      copy_u16(reinterpret_cast<uint16_t*>(hnext + kHaloRunOff), pg, 32 + 2 * hn.n_tb, 32 + 2 * hn.n_tb + 2 * hn.lo_runs);
      copy_u16(reinterpret_cast<uint16_t*>(hnext + kHaloAdcOff), pg, hn.body, hn.body + 4 * ((hn.lo_dig + 2) / 3));
    }
    __syncthreads();

    // ---- 3. decode own page and the two halos into the plane
    if (ok) {
      Seg g{reinterpret_cast<const uint16_t*>(own + 32), h.n_tb,
            reinterpret_cast<const uint16_t*>(own + 32 + 2 * h.n_tb), h.n_runs,
            reinterpret_cast<const uint32_t*>(own + h.body), 0, h.n_dig, kHalo, kFrag * f, true};
      ok = decode_seg(g, np, stride, nw, T, S);
    }
    if (okp) {
      Seg g{reinterpret_cast<const uint16_t*>(hprev), hp.n_tb - hp.hi_tb,
            reinterpret_cast<const uint16_t*>(hprev + kHaloRunOff), hp.n_runs - hp.hi_runs,
            reinterpret_cast<const uint32_t*>(hprev + kHaloAdcOff), hp.hi_dig % 3, hp.n_dig - hp.hi_dig,
            kHalo - kFrag, kFrag * (f - 1), false};
      decode_seg(g, np, stride, nw, T, S);
    }
    if (okn) {
      Seg g{reinterpret_cast<const uint16_t*>(hnext), hn.lo_tb,
            reinterpret_cast<const uint16_t*>(hnext + kHaloRunOff), hn.lo_runs,
            reinterpret_cast<const uint32_t*>(hnext + kHaloAdcOff), 0, hn.lo_dig, kHalo + kFrag, kFrag * (f + 1),
            false};
      decode_seg(g, np, stride, nw, T, S);
    }
    if (!ok && tid == 0) atomicOr(W.err, kErrCorrupt);

    // ---- 4. rank the digits of rows 1..260 (popcount prefix over the bitmap words)
    int ndig = 0;
    {
      const int w0 = tid * wpt, w1 = min(w0 + wpt, nrow_words);
      int c = 0;
      for (int i = w0; i < w1; i++) c += __popc(S.occ[nw + i]);
      unsigned long long tot;
      const unsigned long long pre = block_excl_scan((unsigned long long)c, S.scan, &tot);
      int run = (int)pre;
      for (int i = w0; i < w1; i++) { S.wpre[i] = (uint16_t)run; run += __popc(S.occ[nw + i]); }
      if (tid == 0) S.wpre[nrow_words] = (uint16_t)tot;
      for (int i = w0; i < w1; i++) S.pk[nw + i] = 0u;   // rebuilt by atomicOr below
      ndig = ok ? (int)tot : 0;
    }
    __syncthreads();

    // ---- 5. peak test, one digit per thread (balanced)
    for (int rk = tid; rk < ndig; rk += blockDim.x) {
      const int wi_ = rank_search(S.wpre, nrow_words + 1, rk);
      const uint32_t word = S.occ[nw + wi_];
      const int bit = __fns(word, 0, rk - (int)S.wpre[wi_] + 1);
      const int tt = 1 + wi_ / nw, p = (wi_ % nw) * 32 + bit;
      const int q = S.plane[tt * stride + p];
      if (q >= P.q_peak_min && peak_test(S, stride, nw, np, tt, p, q)) atomicOr(&S.pk[tt * nw + (p >> 5)], 1u << bit);
    }
    __syncthreads();

    // ---- 6. rank the own peaks (rows 3..258) and publish the window's count
    int npk;
    {
      const int w0 = tid * opt, w1 = min(w0 + opt, nown_words);
      int c = 0;
      for (int i = w0; i < w1; i++) c += __popc(S.pk[kHalo * nw + i]);
      unsigned long long tot;
      const unsigned long long pre = block_excl_scan((unsigned long long)c, S.scan, &tot);
      int run = (int)pre;
      for (int i = w0; i < w1; i++) { S.ppre[i] = (uint16_t)run; run += __popc(S.pk[kHalo * nw + i]); }
      if (tid == 0) {
        S.ppre[nown_words] = (uint16_t)tot;
        lookback_publish(W.win_state, (long long)w, tot);
      }
      npk = (int)tot;
    }
    __syncthreads();

    // ---- 7. clusters of the first kStage peaks, staged in shared memory
    const int nst = min(npk, kStage);
    for (int k = tid; k < nst; k += blockDim.x) {
      const int wi_ = rank_search(S.ppre, nown_words + 1, k);
      const uint32_t word = S.pk[kHalo * nw + wi_];
      const int bit = __fns(word, 0, k - (int)S.ppre[wi_] + 1);
      const int tt = kHalo + wi_ / nw, p = (wi_ % nw) * 32 + bit;
      make_cluster(S, stride, nw, np, T, s, r, f, tt, p, G.xrow[r], S.st_rec[k], S.st_xyz[k]);
    }

    // ---- 8. global offset of this window (decoupled look-back)
    if (tid < 32) {
      const unsigned long long base = lookback_wait(W.win_state, (long long)w, (unsigned long long)npk, W.err);
      if (tid == 0) {
        S.scan[33] = base;
        // row starts are clamped to the capacity so that, after an overflow,
        // every later kernel still indexes inside the cluster arrays
        if (f == 0) W.row_start[sr] = (uint32_t)min(base, (unsigned long long)W.cap_cl);
        if (w == n_windows - 1) {
          W.row_start[G.n_sectors * G.n_rows] = (uint32_t)min(base + npk, (unsigned long long)W.cap_cl);
          W.ctr[CTR_NCL] = base + npk;
        }
        if (base + npk > W.cap_cl) atomicOr(W.err, kErrOverflowCl);
      }
    }
    __syncthreads();
    const unsigned long long base = S.scan[33];

    // ---- 9. write out (coalesced), then any peaks beyond the staging buffer
    for (int k = tid; k < npk; k += blockDim.x) {
      const unsigned long long idx = base + k;
      if (idx >= W.cap_cl) break;   // overflow: keep [0, cap) free of gaps, drop the rest
      uint4 rec;
      int4 xyz;
      if (k < kStage) {
        rec = S.st_rec[k];
        xyz = S.st_xyz[k];
      } else {
        const int wi_ = rank_search(S.ppre, nown_words + 1, k);
        const uint32_t word = S.pk[kHalo * nw + wi_];
        const int bit = __fns(word, 0, k - (int)S.ppre[wi_] + 1);
        make_cluster(S, stride, nw, np, T, s, r, f, kHalo + wi_ / nw, (wi_ % nw) * 32 + bit, G.xrow[r], rec, xyz);
      }
      reinterpret_cast<uint4*>(W.clusters)[idx] = rec;
      W.cl_x[idx] = xyz.x;
      W.cl_y[idx] = xyz.y;
      W.cl_z[idx] = xyz.z;
      W.cl_t[idx] = xyz.w;
    }
  }
}

size_t find_smem_bytes(int npmax, int nw) {
  size_t o = ((size_t)kWinT * npmax * 2 + 15) & ~(size_t)15;
  o += 2 * (size_t)kWinT * nw * 4;
  o = (o + 15) & ~(size_t)15;
  o += 2 * kStage * 16 + 2 * kHaloStage + 4 * 16 + 4 * 8 + 34 * 8 + 260 * 4 + 16 * 4;
  o += ((size_t)(kWinT - 2) * nw + 1) * 2 + ((size_t)kFrag * nw + 1) * 2;
  o += 256;
  return o;
}

cudaError_t launch_find(const DevGeom& G, const DevParams& P, const DevWork& W, unsigned int n_windows,
                        int n_sm, cudaStream_t st) {
  size_t sm = find_smem_bytes(G.npmax, G.nw);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_find_clusters, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  unsigned int grid = (unsigned int)min((long long)n_windows, (long long)n_sm * 2);
  if (grid == 0) grid = 1;
  k_find_clusters<<<grid, kFindThreads, sm, st>>>(G, P, W, n_windows);
  return cudaGetLastError();
}

}  // namespace tpc
