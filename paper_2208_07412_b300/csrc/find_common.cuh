// find_common.cuh — pieces shared by the cluster finders (k_find.cu: the fused
// and dense-plane finders and the allocation-free entry point; k_find2.cu: the
// two-pass finder): page header parsing, window coordinates, the block scan and
// the cluster record builder of steps 3-4.
#pragma once
#include "tpc_internal.cuh"

namespace tpc {

constexpr int kPad = 2;                      // empty pads on each side of a plane row

struct PageHdr {
  uint32_t len;
  int n_tb, n_runs, n_dig, sector, row, frag, magic;
  int lo_tb, lo_runs, lo_dig, hi_tb, hi_runs, hi_dig;
  uint32_t body;   // byte offset of the ADC words
};

// Parse and validate a 32-byte page header (from shared or global memory) of
// the page at byte offset `off` of a `pages_bytes` buffer.
__device__ __forceinline__ bool parse_header(const uint4* p, uint64_t off, uint64_t pages_bytes, PageHdr& h) {
  if ((off & 15) || off > pages_bytes || pages_bytes - off < 32) return false;
  const uint4 a = p[0], b = p[1];
  h.len = a.x;
  h.n_tb = a.y & 0xffff; h.n_runs = a.y >> 16;
  h.n_dig = a.z & 0xffff; h.sector = (a.z >> 16) & 0xff; h.row = a.z >> 24;
  h.frag = a.w & 0xffff; h.magic = a.w >> 16;
  h.lo_tb = b.x & 0xffff; h.lo_runs = b.x >> 16; h.lo_dig = b.y & 0xffff;
  h.hi_tb = b.y >> 16; h.hi_runs = b.z & 0xffff; h.hi_dig = b.z >> 16;
  const uint64_t body = (32ull + 2ull * h.n_tb + 2ull * h.n_runs + 3ull) & ~3ull;
  h.body = (uint32_t)body;
  if (h.magic != (int)TPC_ZS_MAGIC || (h.len & 15) || h.len > pages_bytes - off ||
      body + 4ull * ((h.n_dig + 2) / 3) > h.len)
    return false;
  if (h.n_tb > kFrag || h.lo_tb > h.n_tb || h.hi_tb > h.n_tb || h.lo_runs > h.n_runs ||
      h.hi_runs > h.n_runs || h.lo_dig > h.n_dig || h.hi_dig > h.n_dig)
    return false;
  return true;
}

// floor(n / d) for d > 0 and |n / d| < 2^20: a float quotient, corrected
// exactly in integers (its error is far below one).
__device__ __forceinline__ int floordiv32(int n, int d) {
  int q = (int)floorf(__fdividef((float)n, (float)d));
  while (q * d > n) q--;
  while ((q + 1) * d <= n) q++;
  return q;
}
// min(255, R(num, den)) for 0 <= num, 0 < den < 2^31: a float quotient f of
// (2 num + den) / (2 den), whose relative error (operands rounded to float,
// approximate division) stays below 3e-7, i.e. below 1e-4 for quotients up to
// 256; its floor is exact unless f lies within 1e-3 of an integer, where the
// quotient is corrected in 64-bit integers.
__device__ __forceinline__ int round_half_up_sat255(long long num, long long den) {
  const long long n2 = 2 * num + den, d2 = 2 * den;
  const float f = __fdividef((float)n2, (float)d2);
  if (f >= 256.0f) return 255;
  long long q = (long long)f;
  const float fr = f - (float)q;
  if (fr < 1e-3f || fr > 0.999f) {
    while (q > 0 && q * d2 > n2) q--;
    while ((q + 1) * d2 <= n2) q++;
  }
  return (int)min(q, 255LL);
}

// Exclusive block scan of 32-bit counts with one barrier: every warp scans the
// (at most 16) warp totals itself.  sm holds 16 words; two scans with no barrier
// between them must use different sm.
__device__ __forceinline__ uint32_t block_excl_scan32(uint32_t v, uint32_t* sm, uint32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += n;
  }
  if (lane == 31) sm[wid] = inc;
  __syncthreads();
  const uint32_t wv = lane < nw ? sm[lane] : 0u;
  uint32_t wi = wv;
#pragma unroll
  for (int o = 1; o < 16; o <<= 1) {
    const uint32_t n = __shfl_up_sync(0xffffffffu, wi, o);
    if (lane >= o) wi += n;
  }
  const uint32_t before = __shfl_sync(0xffffffffu, wi - wv, wid);
  *total = __shfl_sync(0xffffffffu, wi, nw - 1);
  return before + inc - v;
}

// Window w -> (fragment, row, physical sector) packed f | r << 16 | s << 24,
// computed by one thread and shared (integer divisions by runtime values are
// not worth repeating in every thread).
__device__ __forceinline__ int window_frs(const DevGeom& G, unsigned int w) {
  const int f = (int)(w % (unsigned)G.n_frag);
  const int sr = (int)(w / (unsigned)G.n_frag);
  const int r = sr % G.n_rows, s = (sr / G.n_rows) % G.n_phys;
  return f | (r << 16) | (s << 24);
}

// The record of the cluster of the peak at (tt, p) from its 5x5 charges
// q[dt + 2][dp + 2] and whether another peak lies in the 5x5 (other): the
// inner/outer rule, integer moments, packed 16-byte record and coordinates.
// kW: the moments sum the step-3s weights w instead of q (the rule still reads
// q), and the record is flagged when an included pixel's weight differs.
template <bool kW>
__device__ __forceinline__ void cluster_record_t(const int (&q)[5][5], const int (&w)[5][5], bool other, int np,
                                                 int T, int s, int r, int f, int tt, int p, int xrow, uint4& rec,
                                                 int4& xyz) {
  // included weights summed per pad column (cs) and per time row (rs): the
  // moments are then a few weighted sums of the five of each
  int cs[5] = {0, 0, 0, 0, 0}, rs[5] = {0, 0, 0, 0, 0};
  bool excl = false, split = false;
#pragma unroll
  for (int dt = -2; dt <= 2; dt++) {
#pragma unroll
    for (int dp = -2; dp <= 2; dp++) {
      const int v = q[dt + 2][dp + 2];
      bool inc = true;
      if (dp < -1 || dp > 1 || dt < -1 || dt > 1) {
        const int ip = dp > 0 ? 1 : (dp < 0 ? -1 : 0), it = dt > 0 ? 1 : (dt < 0 ? -1 : 0);
        const int qi = q[it + 2][ip + 2];
        inc = qi > 0 && v <= qi;
        excl |= (!inc && v > 0);
      }
      const int x = kW ? w[dt + 2][dp + 2] : v;
      if (kW) split |= inc && x != v;
      const int xi = inc ? x : 0;
      cs[dp + 2] += xi;
      rs[dt + 2] += xi;
    }
  }
  const int Q = cs[0] + cs[1] + cs[2] + cs[3] + cs[4];
  const int Sp = 2 * (cs[4] - cs[0]) + cs[3] - cs[1], Spp = 4 * (cs[4] + cs[0]) + cs[3] + cs[1];
  const int St = 2 * (rs[4] - rs[0]) + rs[3] - rs[1], Stt = 4 * (rs[4] + rs[0]) + rs[3] + rs[1];
  const int t_in = tt - kHalo;
  const int t = kFrag * f + t_in;
  const int pad_fp = 256 * p + floordiv32(512 * Sp + Q, 2 * Q);
  const int time_fp = 128 * (t_in + 4) + floordiv32(256 * St + Q, 2 * Q);
  const long long QQ = (long long)Q * Q;
  const int vp = round_half_up_sat255(16LL * ((long long)Spp * Q - (long long)Sp * Sp), QQ);
  const int vt = round_half_up_sat255(16LL * ((long long)Stt * Q - (long long)St * St), QQ);
  const int flags = ((p == 0 || p == np - 1 || t == 0 || t == T - 1) ? TPC_CL_EDGE : 0) |
                    (excl ? TPC_CL_EXCLUDED : 0) | (other ? TPC_CL_NEIGHBOUR : 0) | (split ? TPC_CL_SPLIT : 0);
  rec.x = (uint32_t)(pad_fp & 0xffff) | ((uint32_t)(time_fp & 0xffff) << 16);
  rec.y = (uint32_t)q[2][2] | ((uint32_t)min(Q, 65535) << 16);
  rec.z = (uint32_t)vp | ((uint32_t)vt << 8) | ((uint32_t)flags << 16) | ((uint32_t)r << 24);
  rec.w = (uint32_t)t | ((uint32_t)p << 16) | ((uint32_t)s << 24);
  xyz = make_int4(xrow, 2 * (pad_fp - 128 * (np - 1)), 5 * (32768 * f + time_fp - 512), t);
}

__device__ __forceinline__ void cluster_record(const int (&q)[5][5], bool other, int np, int T, int s, int r, int f,
                                               int tt, int p, int xrow, uint4& rec, int4& xyz) {
  cluster_record_t<false>(q, q, other, np, T, s, r, f, tt, p, xrow, rec, xyz);
}

}  // namespace tpc
