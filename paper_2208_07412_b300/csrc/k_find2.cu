// k_find2.cu — the two-pass cluster finder, the pipeline's default for steps
// 1-4 (ZS decode, 3x3 peaks, 5x5 clusters, canonical order).  The paper's
// section "Hardware and data flow" places this first step of the TPC
// reconstruction on the EPN GPUs, after FPGA zero suppression.
//
// Pass 1, k_decode_digits: one warp per page.  Entries, runs and digits are
// walked in chunks of 32 with warp scans (no block barrier): every digit
// becomes one 32-bit word (pad | t_in << 8 | adc << 16) in page order, i.e.
// ascending (time bin, pad), in a span of a digit array the page reserves
// with one atomic.  A table row per window gives the span and the number of
// digits before the time bins H, 64 - H, 64 + H, ..., 192 + H and 256 - H, the
// boundaries of the find units' row ranges for a time halo of H bins (3, or 5
// with charge splitting): the digit index of the first run at or past each,
// stored by the lane that finds it.  Every check of the page format is made
// here; a bad page sets the corruption bit and gets an empty span.
//
// Pass 2, k_find_units: one CTA at a time per unit = (window, 64-bin time
// chunk).  The unit's digits (its 64 time bins with H-bin halos on both sides,
// from the window and, at the fragment edges, its neighbours) go into a
// zero-padded shared plane of 64 + 2H rows (70 rows, 20 KB for 138 pads, instead
// of the 74 KB a whole window needs, so that several CTAs share an SM).  Step 3s
// (charge splitting) needs the peaks up to 4 bins from an own peak, hence the
// values up to 5 bins away: H = 5 there, 3 otherwise.  The peak test runs
// strided over the digits; a peak is marked in the plane (bit 15 of its ADC
// word), which the 5x5 of a cluster reads as "another peak" and step 2b as the
// step-2 peak set; warp ballots rank the own peaks in canonical order into a
// list, over which the clusters are built.  Each unit reserves a span of the
// scratch buffer with one atomic; the unit-count scan and the compaction of
// k_find.cu then place the spans canonically.
#include "find_common.cuh"

namespace tpc {

constexpr int kChunkT = 64;                          // own time bins of a unit
constexpr int kUnitsPerWin = kFrag / kChunkT;        // 4
constexpr int kDecThreads = 256;                     // decode block (8 warps, one page each)
// Time halo of a unit's plane: 3 bins (the 3x3 test of a pixel 2 bins away),
// 5 with step 3s (the peaks up to 4 bins away).
__host__ __device__ constexpr int unit_halo(bool split) { return split ? 5 : 3; }
// Digit counts recorded per window: digits with t_in < bound_of(k, H), k = 0..7.
__device__ __forceinline__ int bound_of(int k, int H) { return kChunkT * ((k + 1) >> 1) + ((k & 1) ? -H : H); }
constexpr uint16_t kPeakBit = 0x8000;                // plane word: a peak of step 2
constexpr uint16_t kDropBit = 0x4000;                // plane word: dropped by step 2b
constexpr uint32_t kAdcMask = 1023u;

__device__ __forceinline__ int warp_incl_scan32(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// The largest lane j < n whose value key (held by lane j, ascending over the
// lanes) is <= x, or 0.  Every lane searches for its own x.
__device__ __forceinline__ int warp_search(int key, int n, int x) {
  int j = 0;
#pragma unroll
  for (int st = 16; st; st >>= 1) {
    const int c = j + st;
    const int kc = __shfl_sync(0xffffffffu, key, c & 31);
    if (c < n && kc <= x) j = c;
  }
  return j;
}

// L2 prefetch of n bytes at p (16-byte aligned, at most 64 KB per instruction).
__device__ __forceinline__ void prefetch_l2_bytes(const void* p, unsigned long long n) {
  for (unsigned long long o = 0; o < n; o += 65536ull) {
    const unsigned m = (unsigned)min(n - o, 65536ull) & ~15u;
    if (m) {
      const size_t ga = __cvta_generic_to_global(reinterpret_cast<const uint8_t*>(p) + o);
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ga), "r"(m) : "memory");
    }
  }
}

constexpr int kDecStage = 4096;                      // bytes of a page body staged per warp

__global__ void __launch_bounds__(kDecThreads, 5) k_decode_digits(DevGeom G, DevWork W, unsigned int n_windows,
                                                                  int H) {
  __shared__ __align__(16) uint8_t stage_all[kDecThreads / 32][kDecStage];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  uint8_t* stage = stage_all[threadIdx.x >> 5];
  const int T = G.n_time_bins;
  while (true) {
    unsigned int w = 0;
    if (lane == 0) w = atomicAdd(W.tickets + TK_DEC, 1u);
    w = __shfl_sync(FULL, w, 0);
    if (w >= n_windows) break;
    const int frs = window_frs(G, w);
    const int f = frs & 0xffff, r = (frs >> 16) & 0xff, s = (frs >> 24) & 0xff;
    const int np = G.npads[r];
    const uint64_t o = W.page_offsets[w];
    PageHdr h;
    bool ok = parse_header(reinterpret_cast<const uint4*>(W.pages + (o <= W.pages_bytes ? o : 0)), o,
                           W.pages_bytes, h) &&
              h.sector == s && h.row == r && h.frag == f;
    unsigned long long base = 0;
    if (ok && lane == 0) base = atomicAdd(&W.ctr[CTR_NDIG], (unsigned long long)h.n_dig);
    base = __shfl_sync(FULL, base, 0);
    // a valid timeframe cannot exceed the array (each digit takes 10 bits of its page)
    if (ok && base + (unsigned long long)h.n_dig > W.cap_dig) ok = false;
    bool bad = !ok;
    int r_cur = 0, d_cur = 0, t_last = -1;
    int carry_t = -1;                     // time bin of the last run seen (boundary crossings)
    // boundary counts (digits before time bin kBound[k]): n_dig unless a run at
    // or past the bin is found, whose first digit index then is the count
    uint16_t* btab = reinterpret_cast<uint16_t*>(W.dtab + 2ull * w + 1);
    if (lane < 8) btab[lane] = (uint16_t)(ok ? h.n_dig : 0);
    __syncwarp();
    if (ok) {
      const uint8_t* pg = W.pages + o;
      // the page body in one round trip: staged in the warp's shared memory
      // (16-byte loads) when it fits, else prefetched into L2 so that its
      // chunks are read from L2 rather than one DRAM round trip after another
      const uint8_t* body = pg + 32;
      const unsigned body_len = h.len - 32u;
      if (body_len <= (unsigned)kDecStage) {
        const uint4* src = reinterpret_cast<const uint4*>(body);
        uint4* dst = reinterpret_cast<uint4*>(stage);
        for (unsigned i = lane; i < body_len / 16u; i += 32u) dst[i] = __ldg(src + i);
        __syncwarp();
        body = stage;
      } else if (lane == 0) {
        prefetch_l2_bytes(body, body_len);
      }
      const uint16_t* ent = reinterpret_cast<const uint16_t*>(body);
      const uint16_t* run = ent + h.n_tb;
      const uint32_t* adc = reinterpret_cast<const uint32_t*>(body + (h.body - 32u));
      uint32_t* out = W.digits + base;
      for (int E = 0; E < h.n_tb && !bad; E += 32) {
        // ---- 32 entries: time bin, run count, first run
        const int e = E + lane, n_ent = min(32, h.n_tb - E);
        int t = 0, nr = 0;
        if (lane < n_ent) {
          const uint32_t v = ent[e];
          t = v & 0xff;
          nr = v >> 8;
        }
        const int tup = __shfl_up_sync(FULL, t, 1);
        const int tp = lane == 0 ? t_last : tup;
        if (lane < n_ent && (nr < 1 || t <= tp || kFrag * f + t >= T)) bad = true;
        const int incl = warp_incl_scan32(nr);
        const int rs = r_cur + incl - nr;                  // first run of entry e
        const int r_end = r_cur + __shfl_sync(FULL, incl, 31);
        t_last = __shfl_sync(FULL, t, n_ent - 1);
        bad = __any_sync(FULL, bad) || r_end > h.n_runs;
        int carry_end = 0, carry_j = -1;
        for (int R = r_cur; R < r_end && !bad; R += 32) {
          // ---- 32 runs: checks, their entry's time bin, digit offsets
          const int ri = R + lane, n_run = min(32, r_end - R);
          int ps = 0, len = 0;
          if (lane < n_run) {
            const uint32_t rv = run[ri];
            ps = rv & 0xff;
            len = rv >> 8;
          }
          const int j = warp_search(rs, n_ent, ri);         // entry of run ri
          const int tr = __shfl_sync(FULL, t, j);
          const int end = ps + len;
          const int pend = __shfl_up_sync(FULL, end, 1), pj = __shfl_up_sync(FULL, j, 1);
          const int prev_end = lane == 0 ? carry_end : pend, prev_j = lane == 0 ? carry_j : pj;
          if (lane < n_run && (len < 1 || end > np || (prev_j == j && ps < prev_end))) bad = true;
          const int tup_r = __shfl_up_sync(FULL, tr, 1);
          const int t_prev_run = lane == 0 ? carry_t : tup_r;
          carry_end = __shfl_sync(FULL, end, 31);
          carry_j = __shfl_sync(FULL, j, 31);
          carry_t = __shfl_sync(FULL, tr, 31);
          const int dinc = warp_incl_scan32(len);
          const int drel = dinc - len;                       // first digit of run ri, within the chunk
          const int n_rd = __shfl_sync(FULL, dinc, 31);
          bad = __any_sync(FULL, bad) || d_cur + n_rd > h.n_dig;
          if (bad) break;
          if (lane < n_run) {
#pragma unroll
            for (int k = 0; k < 8; k++)
              if (t_prev_run < bound_of(k, H) && tr >= bound_of(k, H)) btab[k] = (uint16_t)(d_cur + drel);
          }
          // ---- the chunk's digits, 32 at a time: run by search, ADC from its word
          for (int D = 0; D < n_rd; D += 32) {
            const int dk = D + lane;
            const int k = warp_search(drel, n_run, dk);
            const int ps_k = __shfl_sync(FULL, ps, k), rel_k = __shfl_sync(FULL, drel, k);
            const int t_k = __shfl_sync(FULL, tr, k);
            if (dk < n_rd) {
              const unsigned di = (unsigned)(d_cur + dk);
              const uint32_t wv = adc[di / 3u];
              const uint32_t q = (wv >> (10u * (di % 3u))) & kAdcMask;
              out[di] = (uint32_t)(ps_k + dk - rel_k) | ((uint32_t)t_k << 8) | (q << 16);
            }
          }
          d_cur += n_rd;
        }
        r_cur = r_end;
      }
      if (!bad && (r_cur != h.n_runs || d_cur != h.n_dig)) bad = true;
    }
    __syncwarp();   // the stage is free again
    if (lane == 0) {
      if (bad) atomicOr(W.err, kErrCorrupt);
      const uint32_t n = bad ? 0u : (uint32_t)h.n_dig;
      W.dtab[2ull * w] = make_uint4((uint32_t)base, (uint32_t)(base >> 32), n, 0u);
      if (bad) W.dtab[2ull * w + 1] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

// Digits of window w's table row before boundary k (k = -1: 0; k = 8: all).
__device__ __forceinline__ uint32_t tab_count(const uint4& b, uint32_t n, int k) {
  if (k < 0) return 0u;
  if (k >= 8) return n;
  const uint32_t word = k < 2 ? b.x : (k < 4 ? b.y : (k < 6 ? b.z : b.w));
  return (k & 1) ? word >> 16 : word & 0xffffu;
}

// One unit's digit segments: the previous window's halo, the own chunk, the
// next window's halo.
struct UnitDesc {
  unsigned long long seg_start[3];   // global digit index of each segment's first digit
  int seg_n[3];                      // digits per segment
  int frs, c;                        // window coordinates (f | r << 16 | s << 24), chunk
};

// The descriptor of unit u from the decode table (thread 0 only).
__device__ __forceinline__ void unit_desc(const DevGeom& G, const DevWork& W, unsigned int u, UnitDesc& D) {
  const unsigned int w = u / kUnitsPerWin;
  const int c = (int)(u % kUnitsPerWin);
  const int frs = window_frs(G, w);
  const int f = frs & 0xffff;
  const uint4 a = W.dtab[2ull * w], b = W.dtab[2ull * w + 1];
  const unsigned long long db = a.x | ((unsigned long long)a.y << 32);
  // own digits: time bins [64c - H, 64c + 64 + H) of the window
  const uint32_t lo = tab_count(b, a.z, c == 0 ? -1 : 2 * c - 1);
  const uint32_t hi = tab_count(b, a.z, c == kUnitsPerWin - 1 ? 8 : 2 * c + 2);
  D.seg_start[1] = db + lo;
  D.seg_n[1] = (int)(hi > lo ? hi - lo : 0u);
  D.seg_n[0] = D.seg_n[2] = 0;
  D.seg_start[0] = D.seg_start[2] = 0;
  if (c == 0 && f > 0) {          // the previous window's time bins >= 256 - H
    const uint4 ap = W.dtab[2ull * (w - 1)], bp = W.dtab[2ull * (w - 1) + 1];
    const uint32_t l0 = tab_count(bp, ap.z, 7);
    D.seg_start[0] = (ap.x | ((unsigned long long)ap.y << 32)) + l0;
    D.seg_n[0] = (int)(ap.z > l0 ? ap.z - l0 : 0u);
  }
  if (c == kUnitsPerWin - 1 && f + 1 < G.n_frag) {   // the next window's time bins < H
    const uint4 an = W.dtab[2ull * (w + 1)], bn = W.dtab[2ull * (w + 1) + 1];
    D.seg_start[2] = an.x | ((unsigned long long)an.y << 32);
    D.seg_n[2] = (int)tab_count(bn, an.z, 0);
  }
  D.frs = frs;
  D.c = c;
}

// Unit descriptors, precomputed by k_unit_descs: three 16-byte words per
// unit, (seg_start[0], seg_start[1]), (seg_start[2], seg_n[0], seg_n[1]),
// (seg_n[2], frs, c, 0).
__global__ void k_unit_descs(DevGeom G, DevWork W, unsigned int n_units) {
  for (unsigned int u = blockIdx.x * blockDim.x + threadIdx.x; u < n_units; u += gridDim.x * blockDim.x) {
    UnitDesc D;
    unit_desc(G, W, u, D);
    uint4* q = W.udesc + 3ull * u;
    q[0] = make_uint4((uint32_t)D.seg_start[0], (uint32_t)(D.seg_start[0] >> 32), (uint32_t)D.seg_start[1],
                      (uint32_t)(D.seg_start[1] >> 32));
    q[1] = make_uint4((uint32_t)D.seg_start[2], (uint32_t)(D.seg_start[2] >> 32), (uint32_t)D.seg_n[0],
                      (uint32_t)D.seg_n[1]);
    q[2] = make_uint4((uint32_t)D.seg_n[2], (uint32_t)D.frs, (uint32_t)D.c, 0u);
  }
}

// Digits a thread keeps in registers between the plane build and step 2:
// units with at most kReg * kThreads digits take the register path.
constexpr int kReg = 8;

template <int kThreads>
struct UnitSmem {
  uint4 dq[3][3];                    // descriptor ring: units u, u + G, u + 2G (G = gridDim.x)
  unsigned long long sbase;          // the unit's span of the scratch buffer
  uint32_t total;                    // the unit's own peaks
  uint32_t wtot[2][kThreads / 32];   // per-round warp counts of own peaks (double-buffered)
  uint32_t wcnt[kReg * (kThreads / 32)];   // register path: own peaks per (round, warp), then their prefix
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Step 2 on the plane (bit 15 of a word marks a step-2 peak, bit 14 a peak
// dropped by step 2b; charges are the low 10 bits): neighbours with a lower
// linear index (t * npads + p) must be strictly lower, the others lower or
// equal.
__device__ __forceinline__ bool peak_test(const uint16_t* pl, int L, int ps, int q, int qmin) {
  const uint16_t* u = pl + L - ps;
  const uint16_t* d = pl + L + ps;
  const int lo = max(max((int)(u[-1] & kAdcMask), (int)(u[0] & kAdcMask)),
                     max((int)(u[1] & kAdcMask), (int)(pl[L - 1] & kAdcMask)));
  const int hi = max(max((int)(pl[L + 1] & kAdcMask), (int)(d[-1] & kAdcMask)),
                     max((int)(d[0] & kAdcMask), (int)(d[1] & kAdcMask)));
  return (q >= qmin) & (q > lo) & (q >= hi);
}

// Step 2b for the step-2 peak at plane index L: dropped when a step-2 peak
// with a greater key lies on the ring of its 5x5 window and the inner pixel
// toward it lies less than min_dip below the peak.
__device__ __forceinline__ bool ns_drop_plane(const uint16_t* pl, int L, int ps, int min_dip) {
  const int qc = pl[L] & kAdcMask;
#pragma unroll
  for (int dt = -2; dt <= 2; dt++) {
#pragma unroll
    for (int dp = -2; dp <= 2; dp++) {
      if (dt > -2 && dt < 2 && dp > -2 && dp < 2) continue;   // the ring only
      const uint16_t vn = pl[L + dt * ps + dp];
      if (!(vn & kPeakBit)) continue;
      const int qn = vn & kAdcMask;
      if (qn < qc || (qn == qc && (dt > 0 || (dt == 0 && dp > 0)))) continue;   // not a greater key
      const int it = dt > 0 ? 1 : (dt < 0 ? -1 : 0), ip = dp > 0 ? 1 : (dp < 0 ? -1 : 0);
      if (qc - (int)(pl[L + it * ps + ip] & kAdcMask) < min_dip) return true;
    }
  }
  return false;
}

// L2 prefetch of n digit words from p (widened to whole 16-byte blocks).
__device__ __forceinline__ void prefetch_l2_span(const uint32_t* p, int n) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)15;
  const uintptr_t b = (reinterpret_cast<uintptr_t>(p + n) + 15) & ~(uintptr_t)15;
  prefetch_l2_bytes(reinterpret_cast<const void*>(a), (unsigned long long)(b - a));
}

// Plane row offsets of the three segments: row = t_in + offset.
template <int H>
__device__ __forceinline__ int seg_row_offset(int k, int c) {
  return k == 0 ? H - kFrag : (k == 1 ? H - kChunkT * c : H + kFrag - kChunkT * (kUnitsPerWin - 1));
}

// Step 3s weights of the 5x5 window of the own peak at plane index L (charges
// q, from the plane): w = floor(q(x) q(c) / sum of the owners' charges) when
// the peak c owns x, else 0.  The owners of x are the step-2 peaks of x's 3x3,
// or of its 5x5 when its 3x3 holds none.  A window with no other peak within 4
// pixels keeps w = q.  Reads rows L / ps - 4 .. + 4 (inside the 74-row plane
// for own rows) and pads up to 4 beyond the row, which land on empty padding.
__device__ __forceinline__ void split_weights(const uint16_t* pl, int L, int ps, const int (&q)[5][5],
                                              int (&w)[5][5]) {
  const int qc = q[2][2];
  bool near = false;
  for (int dt = -4; dt <= 4; dt++) {
    const uint16_t* rw = pl + L + dt * ps;
#pragma unroll
    for (int dp = -4; dp <= 4; dp++) near |= (dt | dp) != 0 && (rw[dp] & kPeakBit) != 0;
  }
#pragma unroll
  for (int dt = 0; dt < 5; dt++)
#pragma unroll
    for (int dp = 0; dp < 5; dp++) w[dt][dp] = q[dt][dp];
  if (!near) return;
  for (int dt = -2; dt <= 2; dt++) {
    for (int dp = -2; dp <= 2; dp++) {
      const int v = q[dt + 2][dp + 2];
      if (v == 0) continue;
      const int X = L + dt * ps + dp;
      int s1 = 0;
      for (int a = -1; a <= 1; a++)
        for (int b = -1; b <= 1; b++) {
          const uint16_t y = pl[X + a * ps + b];
          if (y & kPeakBit) s1 += y & kAdcMask;
        }
      int wt;
      if (s1 > 0) {
        wt = (dt >= -1 && dt <= 1 && dp >= -1 && dp <= 1) ? (v * qc) / s1 : 0;
      } else {
        int s2 = 0;   // >= q(c): the peak lies in x's 5x5
        for (int a = -2; a <= 2; a++)
          for (int b = -2; b <= 2; b++) {
            const uint16_t y = pl[X + a * ps + b];
            if (y & kPeakBit) s2 += y & kAdcMask;
          }
        wt = (v * qc) / s2;
      }
      w[dt + 2][dp + 2] = wt;
    }
  }
}

// Units are taken round-robin (unit blockIdx.x + k gridDim.x).  Their
// descriptors come from k_unit_descs two units ahead: lanes 0-2 of warp 0
// copy unit u + 2G's into a ring slot (cp.async) while unit u runs, and thread
// 0 prefetches unit u + G's digits into L2.  Per unit: the plane is built
// from the digits (strided over the threads), step 2 runs strided too, the own
// peaks are ranked in canonical order (digit order) by warp ballots and a
// prefix over (round, warp), and their plane indices listed; the clusters are
// then built strided over that list.  Units of at most kReg * kThreads digits
// (the register path) keep each thread's digits as (plane index, row) words
// in registers between the plane build and step 2, and rank all rounds with
// one prefix; larger units re-read their digits and rank round by round.
template <int kThreads, bool kNs, bool kSplit>
__global__ void __launch_bounds__(kThreads, 1024 / kThreads)
    k_find_units(DevGeom G, DevParams P, DevWork W, unsigned int n_units) {
  constexpr int kH = unit_halo(kSplit);             // time halo of the plane
  constexpr int kURows = kChunkT + 2 * kH;          // plane rows
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ UnitSmem<kThreads> U;
  constexpr int kWarps = kThreads / 32;
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ps = G.npmax + 2 * kPad;                 // plane row stride in pads
  uint16_t* plane = reinterpret_cast<uint16_t*>(smem_raw);
  const int plane_bytes = (kURows * ps * 2 + 15) & ~15;
  const int plane_words16 = plane_bytes / 16;
  uint4* plane16 = reinterpret_cast<uint4*>(smem_raw);
  uint16_t* plist = reinterpret_cast<uint16_t*>(smem_raw + plane_bytes);   // own peaks, canonical order
  for (int i = tid; i < plane_words16; i += kThreads) plane16[i] = make_uint4(0u, 0u, 0u, 0u);
  if (blockIdx.x == 0 && tid == 0) W.ctr[CTR_NWIN] = n_units;
  const int T = G.n_time_bins;
  const unsigned int Gs = gridDim.x;
  // the descriptor ring: units blockIdx.x and blockIdx.x + G in flight
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const unsigned int uk = blockIdx.x + k * Gs;
      if (lane < 3 && uk < n_units) cp_async16(&U.dq[k][lane], W.udesc + 3ull * uk + lane);
      cp_async_commit();
    }
  }
  int slot = 0;
  for (unsigned int u = blockIdx.x; u < n_units; u += Gs) {
    if (wid == 0) {
      const unsigned int u2 = u + 2 * Gs;
      const int s2 = slot == 0 ? 2 : slot - 1;        // (slot + 2) % 3
      if (lane < 3 && u2 < n_units) cp_async16(&U.dq[s2][lane], W.udesc + 3ull * u2 + lane);
      cp_async_commit();
      cp_async_wait1();                                // units u and u + G have landed
    }
    __syncthreads();
    const uint4 q0 = U.dq[slot][0], q1 = U.dq[slot][1], q2 = U.dq[slot][2];
    if (tid == 0 && u + Gs < n_units) {                // unit u + G's digits into L2 meanwhile
      const int s1 = slot == 2 ? 0 : slot + 1;
      const uint4 p0 = U.dq[s1][0], p1 = U.dq[s1][1], p2 = U.dq[s1][2];
      const unsigned long long a0 = p0.x | ((unsigned long long)p0.y << 32);
      const unsigned long long a1 = p0.z | ((unsigned long long)p0.w << 32);
      const unsigned long long a2 = p1.x | ((unsigned long long)p1.y << 32);
      if ((int)p1.z > 0) prefetch_l2_span(W.digits + a0, (int)p1.z);
      if ((int)p1.w > 0) prefetch_l2_span(W.digits + a1, (int)p1.w);
      if ((int)p2.x > 0) prefetch_l2_span(W.digits + a2, (int)p2.x);
    }
    slot = slot == 2 ? 0 : slot + 1;
    const int n0 = (int)q1.z, n01 = n0 + (int)q1.w, n_all = n01 + (int)q2.x;
    const int frs = (int)q2.y, c = (int)q2.z;
    const unsigned long long st0 = q0.x | ((unsigned long long)q0.y << 32);
    const unsigned long long st1 = (q0.z | ((unsigned long long)q0.w << 32)) - n0;
    const unsigned long long st2 = (q1.x | ((unsigned long long)q1.y << 32)) - n01;
    const int of0 = seg_row_offset<kH>(0, c), of1 = seg_row_offset<kH>(1, c), of2 = seg_row_offset<kH>(2, c);
    // digit i of the unit -> (its word, its plane row offset)
    auto digit = [&](int i, int& off) -> uint32_t {
      const unsigned long long g = i < n0 ? st0 + i : (i < n01 ? st1 + i : st2 + i);
      off = i < n0 ? of0 : (i < n01 ? of1 : of2);
      return __ldg(W.digits + g);
    };
    uint32_t total;
    if (n_all <= kReg * kThreads) {
      // ---- register path: build the plane, keeping (L | row << 16) per digit
      uint32_t pk[kReg];
#pragma unroll
      for (int k = 0; k < kReg; k++) {
        pk[k] = FULL;
        const int i = tid + k * kThreads;
        if (i < n_all) {
          int off;
          const uint32_t d = digit(i, off);
          const int row = (int)((d >> 8) & 255u) + off;
          if (row >= 0 && row < kURows) {
            const int L = row * ps + kPad + (int)(d & 255u);
            plane[L] = (uint16_t)(d >> 16);
            pk[k] = (uint32_t)L | ((uint32_t)row << 16);
          }
        }
      }
      __syncthreads();
      // ---- step 2 (rows 1..68): peaks marked, own ones flagged per round
      uint32_t own = 0;
#pragma unroll
      for (int k = 0; k < kReg; k++) {
        if (pk[k] == FULL) continue;
        const int L = (int)(pk[k] & 0xffffu), row = (int)(pk[k] >> 16);
        if (row >= 1 && row <= kURows - 2) {
          const int q = plane[L];
          if (q >= P.q_peak_min && peak_test(plane, L, ps, q, P.q_peak_min)) {
            plane[L] = (uint16_t)(q | kPeakBit);       // only this thread writes this pixel
            if (row >= kH && row < kH + kChunkT) own |= 1u << k;
          }
        }
      }
      if (kNs) {
        __syncthreads();   // every step-2 peak marked: step 2b reads the ring
#pragma unroll
        for (int k = 0; k < kReg; k++) {
          if (!((own >> k) & 1u)) continue;
          const int L = (int)(pk[k] & 0xffffu);
          if (ns_drop_plane(plane, L, ps, P.ns_min_dip)) {
            plane[L] = (uint16_t)(plane[L] | kDropBit);
            own &= ~(1u << k);
          }
        }
      }
      // ---- rank: own peaks per (round, warp), one prefix over them in order
#pragma unroll
      for (int k = 0; k < kReg; k++) {
        const unsigned m = __ballot_sync(FULL, (own >> k) & 1u);
        if (lane == 0) U.wcnt[k * kWarps + wid] = (uint32_t)__popc(m);
      }
      __syncthreads();
      if (wid == 0) {
        uint32_t carry = 0;
#pragma unroll
        for (int j0 = 0; j0 < kReg * kWarps; j0 += 32) {
          const uint32_t v = U.wcnt[j0 + lane];
          const uint32_t inc = (uint32_t)warp_incl_scan32((int)v);
          U.wcnt[j0 + lane] = carry + inc - v;
          carry += __shfl_sync(FULL, inc, 31);
        }
        if (lane == 0) {
          const unsigned long long sb = carry ? atomicAdd(&W.ctr[CTR_SCURSOR], (unsigned long long)carry) : 0ull;
          if (sb + carry > W.cap_cl) atomicOr(W.err, kErrOverflowCl);
          U.sbase = sb;
          U.total = carry;
          W.win_cnt[u] = carry;
          W.win_soff[u] = (uint32_t)min(sb, (unsigned long long)0xffffffffu);
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kReg; k++) {
        const unsigned m = __ballot_sync(FULL, (own >> k) & 1u);
        if ((own >> k) & 1u)
          plist[U.wcnt[k * kWarps + wid] + (uint32_t)__popc(m & ((1u << lane) - 1u))] = (uint16_t)(pk[k] & 0xffffu);
      }
      total = U.total;
    } else {
      // ---- build the plane
      for (int i = tid; i < n_all; i += kThreads) {
        int off;
        const uint32_t d = digit(i, off);
        const int row = (int)((d >> 8) & 255u) + off;
        if (row >= 0 && row < kURows) plane[row * ps + kPad + (int)(d & 255u)] = (uint16_t)(d >> 16);
      }
      __syncthreads();
      // ---- step 2 (rows 1..68), peaks marked; without step 2b the own ones are ranked at once
      uint32_t running = 0;                             // own peaks listed so far (block-uniform)
      int parity = 0;
      for (int base = 0; base < n_all; base += kThreads) {
        const int i = base + tid;
        bool own = false;
        int L = 0;
        if (i < n_all) {
          int off;
          const uint32_t d = digit(i, off);
          const int row = (int)((d >> 8) & 255u) + off;
          if (row >= 1 && row <= kURows - 2) {
            L = row * ps + kPad + (int)(d & 255u);
            const int q = plane[L];
            if (q >= P.q_peak_min && peak_test(plane, L, ps, q, P.q_peak_min)) {
              plane[L] = (uint16_t)(q | kPeakBit);     // only this thread writes this pixel
              own = !kNs && row >= kH && row < kH + kChunkT;
            }
          }
        }
        if (!kNs) {
          const unsigned m = __ballot_sync(FULL, own);
          if (lane == 0) U.wtot[parity][wid] = (uint32_t)__popc(m);
          __syncthreads();
          uint32_t before = running;
#pragma unroll
          for (int k = 0; k < kWarps; k++) {
            const uint32_t v = U.wtot[parity][k];
            before += k < wid ? v : 0u;
            running += v;
          }
          if (own) plist[before + (uint32_t)__popc(m & ((1u << lane) - 1u))] = (uint16_t)L;
          parity ^= 1;
        }
      }
      if (kNs) {
        __syncthreads();   // every step-2 peak marked: step 2b reads the ring
        for (int base = 0; base < n_all; base += kThreads) {
          const int i = base + tid;
          bool own = false;
          int L = 0;
          if (i < n_all) {
            int off;
            const uint32_t d = digit(i, off);
            const int row = (int)((d >> 8) & 255u) + off;
            if (row >= kH && row < kH + kChunkT) {
              L = row * ps + kPad + (int)(d & 255u);
              const uint16_t v = plane[L];
              if (v & kPeakBit) {
                if (ns_drop_plane(plane, L, ps, P.ns_min_dip)) plane[L] = (uint16_t)(v | kDropBit);
                else own = true;
              }
            }
          }
          const unsigned m = __ballot_sync(FULL, own);
          if (lane == 0) U.wtot[parity][wid] = (uint32_t)__popc(m);
          __syncthreads();
          uint32_t before = running;
#pragma unroll
          for (int k = 0; k < kWarps; k++) {
            const uint32_t v = U.wtot[parity][k];
            before += k < wid ? v : 0u;
            running += v;
          }
          if (own) plist[before + (uint32_t)__popc(m & ((1u << lane) - 1u))] = (uint16_t)L;
          parity ^= 1;
        }
      }
      total = running;
      if (tid == 0) {
        const unsigned long long sb = total ? atomicAdd(&W.ctr[CTR_SCURSOR], (unsigned long long)total) : 0ull;
        if (sb + total > W.cap_cl) atomicOr(W.err, kErrOverflowCl);
        U.sbase = sb;
        W.win_cnt[u] = total;
        W.win_soff[u] = (uint32_t)min(sb, (unsigned long long)0xffffffffu);
      }
    }
    __syncthreads();   // list complete, every peak marked, span reserved
    // ---- clusters of the own peaks, strided over the list (canonical order)
    if (total) {
      const unsigned long long sb = U.sbase;
      const int f = frs & 0xffff, r = (frs >> 16) & 0xff, s = (frs >> 24) & 0xff;
      const int np = G.npads[r], xrow = G.xrow[r];
      const int t0 = kChunkT * c - kH;             // time bin (within the window) of plane row 0
      for (uint32_t j = tid; j < total; j += kThreads) {
        const int L = plist[j];
        const int row = L / ps, p = L - row * ps - kPad;
        int q[5][5];
        bool other = false;
#pragma unroll
        for (int dt = 0; dt < 5; dt++)
#pragma unroll
          for (int dp = 0; dp < 5; dp++) {
            const uint16_t x = plane[L + (dt - 2) * ps + dp - 2];
            q[dt][dp] = x & kAdcMask;
            if (dt != 2 || dp != 2) other |= (x & kPeakBit) != 0;
          }
        uint4 rec;
        int4 xyz;
        if (kSplit) {
          int w[5][5];
          split_weights(plane, L, ps, q, w);
          cluster_record_t<true>(q, w, other, np, T, s, r, f, t0 + row + kHalo, p, xrow, rec, xyz);
        } else {
          cluster_record(q, other, np, T, s, r, f, t0 + row + kHalo, p, xrow, rec, xyz);
        }
        const unsigned long long idx = sb + j;
        if (idx < W.cap_cl) reinterpret_cast<uint4*>(W.scratch_cl)[idx] = rec;
      }
    }
    __syncthreads();
    for (int i = tid; i < plane_words16; i += kThreads) plane16[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (wid == 0) asm volatile("cp.async.wait_all;" ::: "memory");
}

// Dynamic shared memory of k_find_units: the plane, then the list of a unit's
// own peaks (at most one per pair of pads of each of its 64 rows).
size_t find2_smem_bytes(int npmax, bool split) {
  return (((size_t)(kChunkT + 2 * unit_halo(split)) * (npmax + 2 * kPad) * 2 + 15) & ~(size_t)15) +
         (size_t)kChunkT * ((npmax + 1) / 2) * 2;
}

template <int kThreads, bool kNs, bool kSplit>
static const void* units_fn() { return (const void*)k_find_units<kThreads, kNs, kSplit>; }

// The instantiation for (threads, step 2b, step 3s).
static const void* units_kernel(int nt, bool ns, bool split) {
  if (nt == 256)
    return split ? (ns ? units_fn<256, true, true>() : units_fn<256, false, true>())
                 : (ns ? units_fn<256, true, false>() : units_fn<256, false, false>());
  return split ? (ns ? units_fn<128, true, true>() : units_fn<128, false, true>())
               : (ns ? units_fn<128, true, false>() : units_fn<128, false, false>());
}

cudaError_t prepare_find2() {
  cudaError_t e = cudaSuccess;
  for (int nt : {128, 256})
    for (int ns = 0; ns < 2; ns++)
      for (int sp = 0; sp < 2; sp++)
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(units_kernel(nt, ns, sp), cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  return e;
}

cudaError_t launch_scan(uint64_t* v, const unsigned long long* n_ptr, unsigned long long cap,
                        unsigned long long* state, unsigned int* ticket, unsigned long long* total, uint32_t* err,
                        int n_sm, cudaStream_t st);
cudaError_t launch_compact(const DevGeom& G, const DevWork& W, unsigned int n_units, int units_per_window, int n_sm,
                           cudaStream_t st);

// Steps 1-4 by the two passes: decode, then find per unit; then the scan of
// the unit counts and the canonical compaction.
cudaError_t launch_find2(const DevGeom& G, const DevParams& P, const DevWork& W, unsigned int n_windows, int n_sm,
                         const LaunchCfg& L, cudaStream_t st, unsigned long long* unit_scan_state, int* launches) {
  const unsigned gd = (unsigned)std::min<unsigned long long>((n_windows + 7ull) / 8ull, (unsigned long long)n_sm * 8);
  const bool split = P.split_charge != 0;
  k_decode_digits<<<gd ? gd : 1, kDecThreads, 0, st>>>(G, W, n_windows, unit_halo(split));
  const unsigned int n_units = n_windows * kUnitsPerWin;
  {
    const unsigned gdesc = (unsigned)std::min<unsigned long long>((n_units + 255ull) / 256ull, (unsigned long long)n_sm * 8);
    k_unit_descs<<<gdesc ? gdesc : 1, 256, 0, st>>>(G, W, n_units);
  }
  const size_t sm = find2_smem_bytes(G.npmax, split);
  const bool ns = P.ns_min_dip > 0;
  const int nt = L.find_threads == 256 ? 256 : 128;
  const void* fn = units_kernel(nt, ns, split);
  // CTAs that are all resident at once (each takes every gridDim.x-th unit)
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, sm) != cudaSuccess || per_sm < 1) per_sm = 1;
  per_sm = std::min(per_sm, L.find_ctas_per_sm);
  const unsigned gu = (unsigned)std::max<unsigned long long>(
      1ull, std::min<unsigned long long>(n_units, (unsigned long long)n_sm * per_sm));
  {
    unsigned int nu = n_units;
    void* args[] = {const_cast<DevGeom*>(&G), const_cast<DevParams*>(&P), const_cast<DevWork*>(&W), &nu};
    cudaError_t le = cudaLaunchKernel(fn, dim3(gu), dim3(nt), args, sm, st);
    if (le != cudaSuccess) return le;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan(reinterpret_cast<uint64_t*>(W.win_cnt), W.ctr + CTR_NWIN, n_units, unit_scan_state,
                  W.tickets + TK_SCAN_W, W.ctr + CTR_NCL, W.err, n_sm, st);
  if (e != cudaSuccess) return e;
  e = launch_compact(G, W, n_units, kUnitsPerWin, n_sm, st);
  *launches += 5;
  return e;
}

}  // namespace tpc
