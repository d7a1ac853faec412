// k_loop.cu — optional looper-leg join (step 9b of the library's definition;
// the paper's section "Hardware and data flow" names the full TPC tracking on
// the EPN GPUs, and a track whose circle lies inside the TPC crosses a sector
// once per turn, each crossing found by steps 5-8 as a track of its own).
//
//   - a track can loop when the circle through its fitted point and direction,
//     with |q/pT| raised by 3 sigma, lies within loop_radius of the beam axis
//     (|centre| + 1/|k| <= loop_radius; centre (x - snp/k, y + cos(phi)/k));
//   - each fit's covariance is scaled by max(1, chi2/ndf);
//   - candidates: tracks A < B (indices) of one (virtual) sector that can
//     loop, fits unflagged, q/pT of one sign; both carried to the larger
//     reference x; m = nearest integer (ties away from zero) to
//     (zeta_B - zeta_A) / S, S = tgl_A 2 pi / |k_A|, 1 <= |m| <= max_turns,
//     tgl_A tgl_B > 0 (zeta advances along every link in the direction of the
//     sign of tgl a chain's legs share, so chains cannot close);
//   - chi2 = d^T (J C_A J^T + C_B)^-1 d, d = s_B - (s_A + m S e_zeta), J the
//     identity plus m 2 pi / |k_A| (zeta, tgl) and -m S / (q/pT)_A (zeta,
//     q/pT); accepted when chi2 <= cut, directed A -> B for m > 0, else B -> A;
//   - a track's next (previous) leg is its outgoing (incoming) accepted pair of
//     least (|m|, chi2, index): a 64-bit atomicMin on |m| << 60 | chi2 bits <<
//     28 | index; f -> g links when g is f's next and f is g's previous.
// The tgl and q/pT components are not changed by the transport nor by J, so
// d_i^2 / (C_A,ii + C_B,ii) for i = tgl, q/pT is a lower bound of the chi2
// (the quadratic form minimised over the other components): a pair above the
// cut on either is rejected before the transport and the 5x5 solve, which
// decides every pair the same way as the full computation.
#include "fit_common.cuh"

namespace tpc {

constexpr unsigned long long kLpIdxMask = (1ull << 28) - 1;

__device__ __forceinline__ unsigned long long n_tracks_lp(const DevWork& W) {
  const unsigned long long n = W.ctr[CTR_NTRK];
  return n < W.cap_ch ? n : W.cap_ch;
}

// Covariance scale of a fit: max(1, chi2/ndf).
__device__ __forceinline__ float cov_scale(float chi2, int ndf) {
  return ndf > 0 && chi2 > (float)ndf ? chi2 / (float)ndf : 1.f;
}

// Farthest distance from the beam axis of the circle through the fitted point
// and direction with |q/pT| raised by 3 sigma; -1 if undefined.
__device__ __forceinline__ float loop_reach(float kfac, const tpc_track& t) {
  const float q = cov_scale(t.chi2, t.ndf);
  const float sq = sqrtf(t.cov[14] * q);
  const float qpt = t.par[4] + (t.par[4] < 0.f ? -3.f : 3.f) * sq;
  const float k = kfac * qpt;
  const float sn = t.par[2];
  if (t.par[4] == 0.f || k == 0.f || !(fabsf(sn) < 1.f)) return -1.f;
  const float cs = sqrtf(1.f - sn * sn);
  const float xc = t.x - sn / k, yc = t.par[0] + cs / k;
  return sqrtf(xc * xc + yc * yc) + 1.f / fabsf(k);
}

__global__ void k_lp_flag(DevGeom G, DevParams P, DevWork W, LoopWork L) {
  const unsigned long long nt = n_tracks_lp(W);
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < nt;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    L.next_key[t] = ~0ull;
    L.prev_key[t] = ~0ull;
    L.next[t] = -1;
    L.prev[t] = -1;
    const tpc_track tr = W.tracks[t];
    uint8_t lp = 0;
    if (!tr.flags) {
      const float r = loop_reach(P.kfac, tr);
      lp = r >= 0.f && r <= L.loop_radius;
    }
    L.loops[t] = lp;
    if (lp) {
      const int vs = vsector_of(G, W, (unsigned)W.trk_first[t], tr.sector);
      atomicAdd(reinterpret_cast<unsigned long long*>(&L.bin_off[vs]), 1ull);
    }
  }
}

// The looping tracks into their virtual sector's bin, each with the first 96
// bytes of its record (state, x, alpha, chi2, covariance, ndf).
__global__ void k_lp_fill(DevGeom G, DevWork W, LoopWork L) {
  const unsigned long long nt = n_tracks_lp(W);
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < nt;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    if (!L.loops[t]) continue;
    const int vs = vsector_of(G, W, (unsigned)W.trk_first[t], W.tracks[t].sector);
    const unsigned long long e = L.bin_off[vs] + atomicAdd(&L.bin_cur[vs], 1u);
    L.ent[e] = (uint32_t)t;
    const uint4* src = reinterpret_cast<const uint4*>(W.tracks + t);
#pragma unroll
    for (int q = 0; q < 6; q++) L.ent_fit[e * 6 + q] = src[q];
  }
}

// State, scaled covariance and reference x of a fit given as its record's
// first 24 words.
struct LegFit {
  float s[5];
  float C[5][5];
  float x;
};

__device__ __forceinline__ void leg_from_words(const float (&w)[24], LegFit& f) {
#pragma unroll
  for (int i = 0; i < 5; i++) f.s[i] = w[i];
  f.x = w[5];
  const float q = cov_scale(w[7], __float_as_int(w[23]));
  int m = 0;
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j <= i; j++) {
      f.C[i][j] = f.C[j][i] = w[8 + m] * q;
      m++;
    }
}

// Carry a leg to x (state and covariance); false if the transport stops.
__device__ __forceinline__ bool carry_leg(float kfac, LegFit& f, float x) {
  if (x == f.x) return true;
  Jac<float> J;
  if (!transport(kfac, f.s, x - f.x, J)) return false;
  float F[5][5];
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j < 5; j++) F[i][j] = i == j ? 1.f : 0.f;
  F[0][2] = J.a; F[0][4] = J.b; F[1][2] = J.e; F[1][3] = J.g; F[1][4] = J.h; F[2][4] = J.m;
  float T[5][5];
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j < 5; j++) {
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < 5; l++) a += F[i][l] * f.C[l][j];
      T[i][j] = a;
    }
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j < 5; j++) {
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < 5; l++) a += T[i][l] * F[j][l];
      f.C[i][j] = a;
    }
  f.x = x;
  return true;
}

// Matching chi2 of legs A (lower index) and B with the signed turn count m;
// a negative value when the pair is no candidate, +inf when a lower bound
// already exceeds the cut.
__device__ float loop_pair(float kfac, const float (&wa)[24], const float (&wb)[24], int max_turns, float cut, int& m) {
  m = 0;
  // the lower bounds on tgl and q/pT (unchanged by the transport and by J)
  {
    const float qa = cov_scale(wa[7], __float_as_int(wa[23])), qb = cov_scale(wb[7], __float_as_int(wb[23]));
    const float d3 = wb[3] - wa[3], d4 = wb[4] - wa[4];
    if (d3 * d3 > cut * (wa[8 + 9] * qa + wb[8 + 9] * qb)) return __int_as_float(0x7f800000);
    if (d4 * d4 > cut * (wa[8 + 14] * qa + wb[8 + 14] * qb)) return __int_as_float(0x7f800000);
  }
  LegFit A, B;
  leg_from_words(wa, A);
  leg_from_words(wb, B);
  const float xr = fmaxf(A.x, B.x);
  if (!carry_leg(kfac, A, xr) || !carry_leg(kfac, B, xr)) return -1.f;
  const float k = kfac * A.s[4];
  if (k == 0.f) return -1.f;
  const float turn = 6.28318530717958648f / fabsf(k);
  const float S = A.s[3] * turn;
  if (S == 0.f) return -1.f;
  const float r = (B.s[1] - A.s[1]) / S;
  if (!(fabsf(r) < (float)max_turns + 0.5f)) return -1.f;
  const float ar = floorf(fabsf(r) + 0.5f);
  m = (int)(r < 0.f ? -ar : ar);
  if (m == 0) return -1.f;
  if (!(A.s[3] * B.s[3] > 0.f)) return -1.f;
  // J C_A J^T: row then column 1 gain j13 (tgl) and j14 (q/pT) multiples
  const float j13 = (float)m * turn, j14 = -(float)m * S / A.s[4];
#pragma unroll
  for (int j = 0; j < 5; j++) A.C[1][j] += j13 * A.C[3][j] + j14 * A.C[4][j];
#pragma unroll
  for (int i = 0; i < 5; i++) A.C[i][1] += j13 * A.C[i][3] + j14 * A.C[i][4];
  float d[5], M[5][5];
#pragma unroll
  for (int i = 0; i < 5; i++) d[i] = B.s[i] - A.s[i];
  d[1] -= (float)m * S;
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j < 5; j++) M[i][j] = A.C[i][j] + B.C[i][j];
  return chi2_spd(M, d);
}

// One warp per looping track A; its lanes take the looping tracks B > A of
// its virtual sector.  The keys are unique (they carry the index), so the
// minima do not depend on which lane finds them.
__global__ void k_lp_pairs(DevGeom G, DevParams P, DevWork W, LoopWork L) {
  const unsigned long long nt = n_tracks_lp(W);
  const int lane = threadIdx.x & 31;
  const unsigned long long wpb = blockDim.x >> 5;
  for (unsigned long long a = blockIdx.x * wpb + (threadIdx.x >> 5); a < nt; a += (unsigned long long)gridDim.x * wpb) {
    if (!L.loops[a]) continue;
    float wa[24];
    {
      const uint4* src = reinterpret_cast<const uint4*>(W.tracks + a);
#pragma unroll
      for (int q = 0; q < 6; q++) {
        const uint4 v = src[q];
        wa[4 * q] = __uint_as_float(v.x);
        wa[4 * q + 1] = __uint_as_float(v.y);
        wa[4 * q + 2] = __uint_as_float(v.z);
        wa[4 * q + 3] = __uint_as_float(v.w);
      }
    }
    const bool pos_a = wa[4] > 0.f;
    const int vs = vsector_of(G, W, (unsigned)W.trk_first[a], W.tracks[a].sector);
    const unsigned long long e0 = L.bin_off[vs], e1 = L.bin_off[vs + 1];
    for (unsigned long long e = e0 + lane; e < e1; e += 32) {
      const unsigned b = L.ent[e];
      if (b <= a) continue;
      float wb[24];
#pragma unroll
      for (int q = 0; q < 6; q++) {
        const uint4 v = L.ent_fit[e * 6 + q];
        wb[4 * q] = __uint_as_float(v.x);
        wb[4 * q + 1] = __uint_as_float(v.y);
        wb[4 * q + 2] = __uint_as_float(v.z);
        wb[4 * q + 3] = __uint_as_float(v.w);
      }
      if ((wb[4] > 0.f) != pos_a) continue;
      int m;
      const float c2 = loop_pair(P.kfac, wa, wb, L.max_turns, L.chi2_cut, m);
      if (!(c2 >= 0.f) || c2 > L.chi2_cut) continue;
      const unsigned f = m > 0 ? (unsigned)a : b, g = m > 0 ? b : (unsigned)a;
      const unsigned long long head = ((unsigned long long)(m < 0 ? -m : m) << 60) |
                                      ((unsigned long long)__float_as_uint(c2) << 28);
      atomicMin(&L.next_key[f], head | g);
      atomicMin(&L.prev_key[g], head | f);
    }
  }
}

__global__ void k_lp_link(DevWork W, LoopWork L) {
  const unsigned long long nt = n_tracks_lp(W);
  unsigned nl = 0;
  for (unsigned long long f = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; f < nt;
       f += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long key = L.next_key[f];
    if (key == ~0ull) continue;
    const unsigned g = (unsigned)(key & kLpIdxMask);
    if ((L.prev_key[g] & kLpIdxMask) == f) {
      L.next[f] = (int)g;
      L.prev[g] = (int)f;
      nl++;
    }
  }
  nl = __reduce_add_sync(0xffffffffu, nl);
  if ((threadIdx.x & 31) == 0 && nl) atomicAdd(&L.ctl[0], (unsigned long long)nl);
}

cudaError_t launch_scan(uint64_t* v, const unsigned long long* n_ptr, unsigned long long cap,
                        unsigned long long* state, unsigned int* ticket, unsigned long long* total, uint32_t* err,
                        int n_sm, cudaStream_t st);

cudaError_t launch_loopers(const DevGeom& G, const DevParams& P, const DevWork& W, const LoopWork& L, int n_sm,
                           cudaStream_t st) {
  unsigned long long g = (W.cap_ch + 255) / 256;
  const unsigned long long gm = (unsigned long long)n_sm * 8;
  if (g > gm) g = gm;
  const unsigned gx = (unsigned)(g ? g : 1);
  k_lp_flag<<<gx, 256, 0, st>>>(G, P, W, L);
  // per-sector counts -> exclusive offsets (n_vs + 1 entries, the last the total)
  cudaError_t e0 = launch_scan(L.bin_off, L.ctl + 1, (unsigned long long)L.n_vs + 1, L.bin_state,
                               reinterpret_cast<unsigned int*>(L.ctl + 2), L.ctl + 3, W.err, n_sm, st);
  if (e0 != cudaSuccess) return e0;
  k_lp_fill<<<gx, 256, 0, st>>>(G, W, L);
  {   // a warp per track: 8 tracks per 256-thread block
    unsigned long long gp = (W.cap_ch + 7) / 8;
    const unsigned long long mp = (unsigned long long)n_sm * 16;
    if (gp > mp) gp = mp;
    k_lp_pairs<<<(unsigned)(gp ? gp : 1), 256, 0, st>>>(G, P, W, L);
  }
  k_lp_link<<<gx, 256, 0, st>>>(W, L);
  return cudaGetLastError();
}

}  // namespace tpc
