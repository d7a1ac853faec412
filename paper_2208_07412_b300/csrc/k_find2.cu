// k_find2.cu — the two-pass cluster finder, the pipeline's default for steps
// 1-4 (ZS decode, 3x3 peaks, 5x5 clusters, canonical order) and the optional
// steps 2b and 3s.  The paper's section "Hardware and data flow" places this
// first step of the TPC reconstruction on the EPN GPUs, after FPGA zero
// suppression.
//
// Pass 1, k_decode_runs: one warp per page.  Entries and runs are walked in
// chunks of 32 with warp scans (no block barrier); every check of the page
// format is made here, and a bad page sets the corruption bit and gets an empty
// span.  Each pad run becomes one 8-byte record (pad, length, time bin, index
// of its first digit in the page) in a span of a run array the page reserves
// with one atomic.  Digits are not touched: their ADCs stay in the page.  A
// table row per window gives the span, the ADC words' offset and the index of
// the first run at or past each of the time bins H, 64 - H, 64 + H, ...,
// 192 + H, 256 - H: the boundaries of the find units' time ranges for a halo of
// H bins (3; 5 with charge splitting, step 3s).
//
// Pass 2, k_find_units: one CTA at a time per unit = (window, 64-bin time
// chunk).  A unit's runs (its 64 time bins with H-bin halos on both sides, from
// the window and, at the fragment edges, its neighbours) are expanded into a
// zero-padded shared plane of 64 + 2H rows (20 KB for 138 pads, so that seven
// CTAs share an SM): one thread per run, its ADCs read from the page (the
// unit's runs and ADC words are prefetched into L2 while the previous unit
// runs; a run's words are then L1 hits after the first).  The expansion also lists
// every digit's plane index in page order (time-major, pad-ascending); step 2
// runs over that list with one thread per digit, marks peaks in the plane (bit
// 15 of the word: what the 5x5 of a cluster reads as "another peak", step 2b as
// the step-2 peak set and step 3s as the owners) and keeps a per-thread bit
// mask of its own peaks, which warp ballots and one prefix rank in canonical
// order.  Units with more digits than the list holds (4096) test every pixel
// of the plane instead, and they and units with more own peaks than their list
// holds (1024) rank the own peaks in pixel order.  Clusters are built over the ranked list; each unit reserves
// a span of the scratch buffer with one atomic, and the unit-count scan and
// the compaction of k_find.cu place the spans canonically.
#include "find_common.cuh"

namespace tpc {

constexpr int kChunkT = 64;                          // own time bins of a unit
constexpr int kUnitsPerWin = kFrag / kChunkT;        // 4
constexpr int kDecThreads = 256;                     // decode block (8 warps, one page each)
constexpr int kDigCap = 4096;                        // digits a unit lists for the digit-driven step 2
constexpr int kPlistCap = 1024;                      // own peaks the list path ranks (else pixel-order ranking)
constexpr int kDescWords = 7;                        // 16-byte words of a unit descriptor
// Time halo of a unit's plane: 3 bins (the 3x3 test of a pixel 2 bins away),
// 5 with step 3s (the peaks up to 4 bins away).
__host__ __device__ constexpr int unit_halo(bool split) { return split ? 5 : 3; }
// Run indices recorded per window: the first run with t_in >= bound_of(k, H), k = 0..7.
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

// L2 prefetch of the bytes [p, p + n), widened to whole 16-byte blocks.
__device__ __forceinline__ void prefetch_l2_range(const void* p, unsigned long long n) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)15;
  const uintptr_t b = (reinterpret_cast<uintptr_t>(p) + n + 15) & ~(uintptr_t)15;
  prefetch_l2_bytes(reinterpret_cast<const void*>(a), (unsigned long long)(b - a));
}

constexpr int kDecStage = 4096;                      // bytes of a page's entries and runs staged per warp

__global__ void __launch_bounds__(kDecThreads, 5) k_decode_runs(DevGeom G, DevWork W, unsigned int n_windows, int H) {
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
    if (ok && lane == 0) base = atomicAdd(&W.ctr[CTR_NRUN], (unsigned long long)h.n_runs);
    base = __shfl_sync(FULL, base, 0);
    // a valid timeframe cannot exceed the array (each run takes more than 3 bytes of its page)
    if (ok && base + (unsigned long long)h.n_runs > W.cap_runs) ok = false;
    bool bad = !ok;
    int r_cur = 0, d_cur = 0, t_last = -1;
    // boundary run indices: n_runs unless an entry at or past the bin is found,
    // whose first run then is the index
    uint16_t* btab = reinterpret_cast<uint16_t*>(W.dtab + 3ull * w + 1);
    if (lane < 8) btab[lane] = (uint16_t)(ok ? h.n_runs : 0);
    __syncwarp();
    if (ok) {
      const uint8_t* pg = W.pages + o;
      // entries and runs in one round trip: staged in the warp's shared memory
      // (16-byte loads, within the page) when they fit, else prefetched into L2
      const uint8_t* body = pg + 32;
      const unsigned meta_len = (h.body - 32u + 15u) & ~15u;
      if (meta_len <= (unsigned)kDecStage) {
        const uint4* src = reinterpret_cast<const uint4*>(body);
        uint4* dst = reinterpret_cast<uint4*>(stage);
        for (unsigned i = lane; i < meta_len / 16u; i += 32u) dst[i] = __ldg(src + i);
        __syncwarp();
        body = stage;
      } else if (lane == 0) {
        prefetch_l2_bytes(body, meta_len);
      }
      const uint16_t* ent = reinterpret_cast<const uint16_t*>(body);
      const uint16_t* run = ent + h.n_tb;
      uint2* out = W.runs + base;
      for (int E = 0; E < h.n_tb && !bad; E += 32) {
        // ---- 32 entries: time bin, run count, first run; the units' boundaries
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
        if (bad) break;
        if (lane < n_ent) {
#pragma unroll
          for (int k = 0; k < 8; k++) {
            const int bk = bound_of(k, H);
            if (tp < bk && t >= bk) btab[k] = (uint16_t)rs;
          }
        }
        int carry_end = 0, carry_j = -1;
        for (int R = r_cur; R < r_end && !bad; R += 32) {
          // ---- 32 runs: their entry's time bin, checks, first digits, records
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
          carry_end = __shfl_sync(FULL, end, 31);
          carry_j = __shfl_sync(FULL, j, 31);
          const int dinc = warp_incl_scan32(len);
          const int n_rd = __shfl_sync(FULL, dinc, 31);
          bad = __any_sync(FULL, bad) || d_cur + n_rd > h.n_dig;
          if (bad) break;
          if (lane < n_run)
            out[ri] = make_uint2((uint32_t)ps | ((uint32_t)len << 8) | ((uint32_t)tr << 16),
                                 (uint32_t)(d_cur + dinc - len));
          d_cur += n_rd;
        }
        r_cur = r_end;
      }
      if (!bad && (r_cur != h.n_runs || d_cur != h.n_dig)) bad = true;
    }
    __syncwarp();   // the stage is free again
    if (lane == 0) {
      if (bad) atomicOr(W.err, kErrCorrupt);
      const uint32_t n = bad ? 0u : (uint32_t)h.n_runs;
      const unsigned long long adc = ok ? o + h.body : 0ull;
      W.dtab[3ull * w] = make_uint4((uint32_t)base, (uint32_t)(base >> 32), n, 0u);
      if (bad) W.dtab[3ull * w + 1] = make_uint4(0u, 0u, 0u, 0u);
      W.dtab[3ull * w + 2] = make_uint4((uint32_t)adc, (uint32_t)(adc >> 32), 0u, 0u);
    }
  }
}

// Run index of window table row b before boundary k (k = -1: 0; k = 8: all n).
__device__ __forceinline__ uint32_t tab_run(const uint4& b, uint32_t n, int k) {
  if (k < 0) return 0u;
  if (k >= 8) return n;
  const uint32_t word = k < 2 ? b.x : (k < 4 ? b.y : (k < 6 ? b.z : b.w));
  return (k & 1) ? word >> 16 : word & 0xffffu;
}

// Unit descriptors, precomputed by k_unit_descs: per segment k (the previous
// window's halo, the own window, the next window's halo) two 16-byte words
//   (first run lo, hi, runs, index in the page of the first digit dA)
//   (first ADC word lo, hi (index into the pages as 32-bit words), ADC words, digits)
// then (frs, chunk, digits of all segments, ADC words of all segments).
__global__ void k_unit_descs(DevGeom G, DevWork W, unsigned int n_units) {
  for (unsigned int u = blockIdx.x * blockDim.x + threadIdx.x; u < n_units; u += gridDim.x * blockDim.x) {
    const unsigned int w = u / kUnitsPerWin;
    const int c = (int)(u % kUnitsPerWin);
    const int frs = window_frs(G, w);
    const int f = frs & 0xffff;
    uint4* q = W.udesc + (unsigned long long)kDescWords * u;
    uint32_t tot_d = 0, tot_w = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      // segment 0: the previous window's time bins >= 256 - H; 1: own time bins
      // [64c - H, 64c + 64 + H); 2: the next window's time bins < H
      const bool have = k == 1 || (k == 0 && c == 0 && f > 0) || (k == 2 && c == kUnitsPerWin - 1 && f + 1 < G.n_frag);
      uint32_t n = 0, dA = 0, nd = 0, nw = 0;
      unsigned long long start = 0, aw = 0;
      if (have) {
        const unsigned long long ws = (unsigned long long)w + k - 1;
        const uint4 a = W.dtab[3ull * ws], b = W.dtab[3ull * ws + 1], cc = W.dtab[3ull * ws + 2];
        uint32_t lo, hi;
        if (k == 0) { lo = tab_run(b, a.z, 2 * kUnitsPerWin - 1); hi = a.z; }
        else if (k == 1) {
          lo = tab_run(b, a.z, c == 0 ? -1 : 2 * c - 1);
          hi = tab_run(b, a.z, c == kUnitsPerWin - 1 ? 8 : 2 * c + 2);
        } else { lo = 0; hi = tab_run(b, a.z, 0); }
        if (hi > lo) {
          n = hi - lo;
          start = (a.x | ((unsigned long long)a.y << 32)) + lo;
          const uint2 r0 = W.runs[start], r1 = W.runs[start + n - 1];
          dA = r0.y;
          const uint32_t dB = r1.y + ((r1.x >> 8) & 255u);
          nd = dB - dA;
          nw = (dB - 1u) / 3u - dA / 3u + 1u;
          aw = ((cc.x | ((unsigned long long)cc.y << 32)) >> 2) + dA / 3u;
        }
      }
      q[2 * k] = make_uint4((uint32_t)start, (uint32_t)(start >> 32), n, dA);
      q[2 * k + 1] = make_uint4((uint32_t)aw, (uint32_t)(aw >> 32), nw, nd);
      tot_d += nd;
      tot_w += nw;
    }
    q[6] = make_uint4((uint32_t)frs, (uint32_t)c, tot_d, tot_w);
  }
}

template <int kThreads>
struct UnitSmem {
  uint4 dq[3][kDescWords];           // descriptor ring: units u, u + G, u + 2G (G = gridDim.x)
  unsigned long long sbase;          // the unit's span of the scratch buffer
  uint32_t total;                    // the unit's own peaks
  uint32_t wcnt[2][32 * (kThreads / 32)];   // own peaks per (round, warp) of a batch of at most 32 rounds
};

// Ranking of own peaks in canonical order.  A batch is up to 32 rounds of
// kThreads items in canonical order (item tid + k kThreads of round k); bit k
// of a thread's mask own marks an own peak.  rank_count stores the own peaks
// per (round, warp); after a barrier, rank_place has every warp scan those
// counts itself and list its own peaks at base + their rank (item_L(k) gives
// the plane index of round k's item).  Returns the batch's own peaks.
template <int kThreads>
__device__ __forceinline__ void rank_count(uint32_t own, int nr, uint32_t* wcnt) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < nr; k++) {
    const unsigned m = __ballot_sync(0xffffffffu, (own >> k) & 1u);
    if (lane == 0) wcnt[k * (kThreads / 32) + wid] = (uint32_t)__popc(m);
  }
}

template <int kThreads, typename ItemL>
__device__ __forceinline__ uint32_t rank_place(uint32_t own, int nr, const uint32_t* wcnt, uint32_t base,
                                               uint16_t* plist, ItemL item_L) {
  constexpr int kWarps = kThreads / 32;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t carry = 0;
  for (int j0 = 0; j0 < nr * kWarps; j0 += 32) {
    const bool in = j0 + lane < nr * kWarps;
    const uint32_t v = in ? wcnt[j0 + lane] : 0u;
    const uint32_t inc = (uint32_t)warp_incl_scan32((int)v);
    const uint32_t excl = base + carry + inc - v;      // own peaks before (round, warp) j0 + lane
    // this warp's rounds k with k * kWarps + wid in [j0, j0 + 32)
    for (int k = (j0 + kWarps - 1 - wid) / kWarps; k < nr && k * kWarps + wid < j0 + 32; k++) {
      const uint32_t before = __shfl_sync(FULL, excl, k * kWarps + wid - j0);
      const unsigned m = __ballot_sync(FULL, (own >> k) & 1u);
      if ((own >> k) & 1u) plist[before + (uint32_t)__popc(m & ((1u << lane) - 1u))] = (uint16_t)item_L(k);
    }
    carry += __shfl_sync(FULL, inc, 31);
  }
  return carry;
}

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

// Plane row offsets of the three segments: row = t_in + offset.
template <int H>
__device__ __forceinline__ int seg_row_offset(int k, int c) {
  return k == 0 ? H - kFrag : (k == 1 ? H - kChunkT * c : H + kFrag - kChunkT * (kUnitsPerWin - 1));
}

// Units are taken round-robin (unit blockIdx.x + k gridDim.x).  Their
// descriptors come from k_unit_descs two units ahead: lanes 0-6 of warp 0
// copy unit u + 2G's into a ring slot (cp.async) while unit u runs, and thread
// 0 prefetches unit u + G's runs and ADC words into L2.  Per unit: the runs
// are expanded into the plane and the digit list, step 2 runs over the list
// (or over every pixel: dense path), the own peaks are ranked, and the
// clusters built from the ranked list.  Shared memory after the plane: the
// digit list and the list path's own peaks, or the dense path's own peaks.
template <int kThreads, bool kNs, bool kSplit>
__global__ void __launch_bounds__(kThreads, 896 / kThreads)
    k_find_units(DevGeom G, DevParams P, DevWork W, unsigned int n_units) {
  constexpr int kH = unit_halo(kSplit);             // time halo of the plane
  constexpr int kURows = kChunkT + 2 * kH;          // plane rows
  static_assert(kDigCap / kThreads <= 32, "one own-peak mask bit per list round");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ UnitSmem<kThreads> U;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ps = G.npmax + 2 * kPad;                 // plane row stride in pads
  const int plane_bytes = (kURows * ps * 2 + 15) & ~15;
  const int plane_words16 = plane_bytes / 16;
  uint16_t* plane = reinterpret_cast<uint16_t*>(smem_raw);
  uint4* plane16 = reinterpret_cast<uint4*>(smem_raw);
  uint16_t* dl = reinterpret_cast<uint16_t*>(smem_raw + plane_bytes);   // the digits' plane indices
  uint16_t* plist_l = dl + kDigCap;                                        // list path: own peaks, canonical order
  uint16_t* plist_d = dl;                                                  // dense path: the same
  const uint32_t* pages32 = reinterpret_cast<const uint32_t*>(W.pages);
  for (int i = tid; i < plane_words16; i += kThreads) plane16[i] = make_uint4(0u, 0u, 0u, 0u);
  if (blockIdx.x == 0 && tid == 0) W.ctr[CTR_NWIN] = n_units;
  const int T = G.n_time_bins;
  const unsigned int Gs = gridDim.x;
  // the descriptor ring: units blockIdx.x and blockIdx.x + G in flight
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const unsigned int uk = blockIdx.x + k * Gs;
      if (lane < kDescWords && uk < n_units)
        cp_async16(&U.dq[k][lane], W.udesc + (unsigned long long)kDescWords * uk + lane);
      cp_async_commit();
    }
  }
  int slot = 0;
  for (unsigned int u = blockIdx.x; u < n_units; u += Gs) {
    if (wid == 0) {
      const unsigned int u2 = u + 2 * Gs;
      const int s2 = slot == 0 ? 2 : slot - 1;        // (slot + 2) % 3
      if (lane < kDescWords && u2 < n_units)
        cp_async16(&U.dq[s2][lane], W.udesc + (unsigned long long)kDescWords * u2 + lane);
      cp_async_commit();
      cp_async_wait1();                                // units u and u + G have landed
    }
    __syncthreads();
    // ---- the unit's segments
    unsigned long long rstart[3], aw[3];
    uint32_t nrun[3], dA[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const uint4 a = U.dq[slot][2 * k], b = U.dq[slot][2 * k + 1];
      rstart[k] = a.x | ((unsigned long long)a.y << 32);
      nrun[k] = a.z;
      dA[k] = a.w;
      aw[k] = b.x | ((unsigned long long)b.y << 32);
    }
    const uint4 q6 = U.dq[slot][6];
    const int frs = (int)q6.x, c = (int)q6.y;
    const uint32_t n_dig = q6.z;
    const uint32_t doff1 = U.dq[slot][1].w, doff2 = doff1 + U.dq[slot][3].w;   // list offsets of segments 1, 2
    const uint32_t roff1 = nrun[0], roff2 = nrun[0] + nrun[1], n_runs = roff2 + nrun[2];
    if (wid == kThreads / 32 - 1 && lane < 6 && u + Gs < n_units) {
      // unit u + G's runs (lanes 0-2) and ADC words (lanes 3-5) into L2
      // meanwhile, one segment per lane of the last warp
      const int s1 = slot == 2 ? 0 : slot + 1;
      const int k = lane % 3;
      const uint4 a = U.dq[s1][2 * k], b = U.dq[s1][2 * k + 1];
      if (a.z) {
        if (lane < 3) prefetch_l2_range(W.runs + (a.x | ((unsigned long long)a.y << 32)), 8ull * a.z);
        else prefetch_l2_range(pages32 + (b.x | ((unsigned long long)b.y << 32)), 4ull * b.z);
      }
    }
    slot = slot == 2 ? 0 : slot + 1;
    const bool list = n_dig <= (uint32_t)kDigCap;     // block-uniform
    bool pixel_rank = !list;                           // rank by pixel order (block-uniform)
    // ---- build: one thread per run; its digits go into the plane (and the list)
    for (uint32_t i = tid; i < n_runs; i += kThreads) {
      const int k = i < roff1 ? 0 : (i < roff2 ? 1 : 2);
      const uint32_t ri = i - (k == 0 ? 0u : (k == 1 ? roff1 : roff2));
      const uint2 rec = __ldg(W.runs + (k == 0 ? rstart[0] : (k == 1 ? rstart[1] : rstart[2])) + ri);
      const int p0 = (int)(rec.x & 255u), len = (int)((rec.x >> 8) & 255u);
      const int row = (int)((rec.x >> 16) & 255u) + seg_row_offset<kH>(k, c);
      if (row < 0 || row >= kURows) continue;          // cannot happen for a decoded page
      const int L0 = row * ps + kPad + p0;
      const uint32_t d0 = rec.y;
      const uint32_t dk = k == 0 ? dA[0] : (k == 1 ? dA[1] : dA[2]);
      uint32_t sub = d0 % 3u;
      const uint32_t* src = pages32 + (k == 0 ? aw[0] : (k == 1 ? aw[1] : aw[2])) + (d0 / 3u - dk / 3u);
      uint32_t word = __ldg(src);
      if (list) {
        uint16_t* dst = dl + (k == 0 ? 0u : (k == 1 ? doff1 : doff2)) + (d0 - dk);
        for (int j = 0; j < len; j++) {
          if (j > 0 && sub == 0) word = __ldg(++src);
          plane[L0 + j] = (uint16_t)((word >> (10u * sub)) & kAdcMask);
          dst[j] = (uint16_t)(L0 + j);
          sub = sub == 2u ? 0u : sub + 1u;
        }
      } else {
        for (int j = 0; j < len; j++) {
          if (j > 0 && sub == 0) word = __ldg(++src);
          plane[L0 + j] = (uint16_t)((word >> (10u * sub)) & kAdcMask);
          sub = sub == 2u ? 0u : sub + 1u;
        }
      }
    }
    __syncthreads();   // plane and digit list complete
    const int qmin = P.q_peak_min;
    const int test_lo = ps, test_hi = (kURows - 1) * ps;          // rows 1 .. kURows - 2
    const int own_lo = kH * ps, own_hi = (kH + kChunkT) * ps;     // own rows
    uint32_t total = 0;
    if (list) {
      // ---- step 2 over the digit list: peaks marked, own ones flagged per round
      const int nr = (int)((n_dig + kThreads - 1) / kThreads);
      uint32_t own = 0;
      for (int k = 0; k < nr; k++) {
        const uint32_t i = tid + (uint32_t)k * kThreads;
        if (i < n_dig) {
          const int L = dl[i];
          if (L >= test_lo && L < test_hi) {
            const int q = plane[L];                     // only this thread marks this pixel
            if (q >= qmin && peak_test(plane, L, ps, q, qmin)) {
              plane[L] = (uint16_t)(q | kPeakBit);
              if (L >= own_lo && L < own_hi) own |= 1u << k;
            }
          }
        }
      }
      if (kNs) {
        __syncthreads();   // every step-2 peak marked: step 2b reads the ring
        for (int k = 0; k < nr; k++) {
          if (!((own >> k) & 1u)) continue;
          const int L = dl[tid + (uint32_t)k * kThreads];
          if (ns_drop_plane(plane, L, ps, P.ns_min_dip)) {
            plane[L] = (uint16_t)(plane[L] | kDropBit);
            own &= ~(1u << k);
          }
        }
      }
      // ---- rank: one batch (nr <= 32 rounds), unless the own peaks overflow their list
      rank_count<kThreads>(own, nr, U.wcnt[0]);
      __syncthreads();
      uint32_t cnt = 0;
      for (int j = lane; j < nr * (kThreads / 32); j += 32) cnt += U.wcnt[0][j];
#pragma unroll
      for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      if (cnt <= (uint32_t)kPlistCap)
        total = rank_place<kThreads>(own, nr, U.wcnt[0], 0u, plist_l,
                                     [&](int k) { return (int)dl[tid + (uint32_t)k * kThreads]; });
      else
        pixel_rank = true;   // block-uniform: every warp summed the same counts
    } else {
      // ---- dense path: step 2 on every pixel of rows 1 .. kURows - 2
      const int np = G.npads[(frs >> 16) & 0xff];
      const int n_test = (kURows - 2) * np;
      for (int i = tid; i < n_test; i += kThreads) {
        const int row = 1 + i / np, p = i - (row - 1) * np;
        const int L = row * ps + kPad + p;
        const int q = plane[L];
        if (q >= qmin && peak_test(plane, L, ps, q, qmin)) plane[L] = (uint16_t)(q | kPeakBit);
      }
      __syncthreads();   // every step-2 peak marked
    }
    if (pixel_rank) {
      // ---- rank the own pixels' peaks (step 2b decided inline; again, with
      // the same result, for peaks the list path has decided) in batches of 32
      // rounds of kThreads pixels, canonical order.  The batches alternate
      // between the two count buffers, starting with the one the list path
      // did not use, so one barrier per batch suffices.
      const int np = G.npads[(frs >> 16) & 0xff];
      const int n_own = kChunkT * np;
      auto pix_L = [&](int i) { const int row = kH + i / np; return row * ps + kPad + (i - (row - kH) * np); };
      uint32_t running = 0;                             // own peaks listed so far (block-uniform)
      int parity = 1;
      for (int B = 0; B < n_own; B += 32 * kThreads) {
        const int nrb = min(32, (n_own - B + kThreads - 1) / kThreads);
        uint32_t own = 0;
        for (int k = 0; k < nrb; k++) {
          const int i = B + k * kThreads + tid;
          if (i < n_own) {
            const int L = pix_L(i);
            const uint16_t v = plane[L];
            if (v & kPeakBit) {
              if (kNs && ns_drop_plane(plane, L, ps, P.ns_min_dip)) plane[L] = (uint16_t)(v | kDropBit);
              else own |= 1u << k;
            }
          }
        }
        rank_count<kThreads>(own, nrb, U.wcnt[parity]);
        __syncthreads();
        running += rank_place<kThreads>(own, nrb, U.wcnt[parity], running, plist_d,
                                        [&](int k) { return pix_L(B + k * kThreads + tid); });
        parity ^= 1;
      }
      total = running;
    }
    if (tid == 0) {
      const unsigned long long sb = total ? atomicAdd(&W.ctr[CTR_SCURSOR], (unsigned long long)total) : 0ull;
      if (sb + total > W.cap_cl) atomicOr(W.err, kErrOverflowCl);
      U.sbase = sb;
      W.win_cnt[u] = total;
      W.win_soff[u] = (uint32_t)min(sb, (unsigned long long)0xffffffffu);
    }
    __syncthreads();   // list complete, every peak marked, span reserved
    // ---- clusters of the own peaks, strided over the list (canonical order)
    if (total) {
      const uint16_t* plist = pixel_rank ? plist_d : plist_l;
      const unsigned long long sb = U.sbase;
      const int f = frs & 0xffff, r = (frs >> 16) & 0xff, s = (frs >> 24) & 0xff;
      const int np = G.npads[r], xrow = G.xrow[r];
      const int t0 = kChunkT * c - kH;             // time bin (within the window) of plane row 0
      for (uint32_t j = tid; j < total; j += kThreads) {
        const int L = plist[j];
        const int row = L / ps, p = L - row * ps - kPad;
        int q[5][5];
        unsigned ring = 0;                             // the other 24 words ORed: a peak among them?
#pragma unroll
        for (int dt = 0; dt < 5; dt++)
#pragma unroll
          for (int dp = 0; dp < 5; dp++) {
            const uint16_t x = plane[L + (dt - 2) * ps + dp - 2];
            q[dt][dp] = x & kAdcMask;
            if (dt != 2 || dp != 2) ring |= x;
          }
        const bool other = (ring & kPeakBit) != 0;
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
    // the plane back to zero: only the listed digits' pixels were written on
    // the list path (the list is intact unless the pixel-order ranking used its room)
    if (!pixel_rank) {
      for (uint32_t i = tid; i < n_dig; i += kThreads) plane[dl[i]] = 0;
    } else {
      for (int i = tid; i < plane_words16; i += kThreads) plane16[i] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  if (wid == 0) asm volatile("cp.async.wait_all;" ::: "memory");
}

// Dynamic shared memory of k_find_units: the plane, then either the digit
// list (kDigCap entries) and the own peaks of the list path (kPlistCap), or
// the own peaks ranked by pixel order (at most one per pair of pads of each of
// 64 rows).
size_t find2_smem_bytes(int npmax, bool split) {
  const size_t plane = ((size_t)(kChunkT + 2 * unit_halo(split)) * (npmax + 2 * kPad) * 2 + 15) & ~(size_t)15;
  const size_t dense_peaks = (size_t)kChunkT * ((npmax + 1) / 2) * 2;
  const size_t r = std::max(dense_peaks, (size_t)(kDigCap + kPlistCap) * 2);
  return plane + ((r + 15) & ~(size_t)15);
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
        if (e == cudaSuccess) {
          e = cudaFuncSetAttribute(units_kernel(nt, ns, sp), cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
          // all of the unified L1 / shared storage as shared memory: seven CTAs of ~32 KB per SM
          if (e == cudaSuccess)
            e = cudaFuncSetAttribute(units_kernel(nt, ns, sp), cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        }
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
  k_decode_runs<<<gd ? gd : 1, kDecThreads, 0, st>>>(G, W, n_windows, unit_halo(split));
  unsigned int n_units = n_windows * kUnitsPerWin;
  {
    const unsigned gdesc = (unsigned)std::min<unsigned long long>((n_units + 255ull) / 256ull, (unsigned long long)n_sm * 8);
    k_unit_descs<<<gdesc ? gdesc : 1, 256, 0, st>>>(G, W, n_units);
  }
  const bool ns = P.ns_min_dip > 0;
  const int nt = L.find_threads == 256 ? 256 : 128;
  const size_t sm = find2_smem_bytes(G.npmax, split);
  const void* fn = units_kernel(nt, ns, split);
  // CTAs that are all resident at once (each takes every gridDim.x-th unit)
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, sm) != cudaSuccess || per_sm < 1) per_sm = 1;
  per_sm = std::min(per_sm, L.find_ctas_per_sm);
  const unsigned gu = (unsigned)std::max<unsigned long long>(
      1ull, std::min<unsigned long long>(n_units, (unsigned long long)n_sm * per_sm));
  {
    void* args[] = {const_cast<DevGeom*>(&G), const_cast<DevParams*>(&P), const_cast<DevWork*>(&W), &n_units};
    cudaError_t le = cudaLaunchKernel(fn, dim3(gu), dim3(nt), args, sm, st);
    if (le != cudaSuccess) return le;
  }
  cudaError_t e = launch_scan(reinterpret_cast<uint64_t*>(W.win_cnt), W.ctr + CTR_NWIN, n_units, unit_scan_state,
                              W.tickets + TK_SCAN_W, W.ctr + CTR_NCL, W.err, n_sm, st);
  if (e != cudaSuccess) return e;
  e = launch_compact(G, W, n_units, kUnitsPerWin, n_sm, st);
  *launches += 5;
  return e;
}

}  // namespace tpc
