// k_xsec.cu — optional cross-sector merge (step 9 of the library's definition;
// the paper's section "Hardware and data flow" names the full TPC tracking on
// the EPN GPUs, and joining the pieces of a track that crosses a sector border
// is this library's last step of it).
//
//   - a track exits through the +y (-y) edge of its sector when its outermost
//     cluster lies within E = edge_cm / u of that edge of the pad plane
//     (|Y| >= 256 (npads - 1) - E, integer u); it enters through an edge when its
//     innermost cluster does;
//   - candidate pairs: A exiting through +y (-y) of sector s, B entering through
//     -y (+y) of the neighbouring sector s+1 (s-1) of the same side, A's
//     outermost row below B's innermost row, neither fit flagged;
//   - B's fitted state is rotated into A's frame (about the beam axis) and
//     transported to A's reference x; chi2 = d^T (C_A + J C_B J^T)^-1 d;
//   - mutual best pairs with chi2 <= chi2_cut link (64-bit atomicMin on
//     (chi2 bits << 32 | index): ties to the lower index);
//   - each chain of linked pieces becomes one track, refitted over all its
//     clusters in FP32 (U D U^T factors, FP64 redo on a failed PD check) with
//     the state and the factors rotated into a piece's frame before its first
//     cluster is reached.
// Rotation by delta = alpha_old - alpha_new of a state at x: the point (x, y)
// maps to (x cos d - y sin d, x sin d + y cos d), the direction gains d; its
// first-order Jacobian at the rotated reference (the point moves with y by
// dx' = -sin d dy and is carried back along the helix): dy' = (cos d + tan(phi')
// sin d) dy, dzeta' = dzeta + (tgl / cos(phi')) sin d dy, dsnp' = (cos d - sin d
// snp / cos(phi)) dsnp + k sin d dy.  The factors follow by W = R U and a
// modified weighted Gram-Schmidt re-triangularisation of W D W^T.
#include "fit_common.cuh"

namespace tpc {


__device__ __forceinline__ unsigned long long n_tracks_x(const DevWork& W) {
  const unsigned long long n = W.ctr[CTR_NTRK];
  return n < W.cap_ch ? n : W.cap_ch;
}

__device__ __forceinline__ int side_code(int Y, int np, int E) {
  const int hw = 256 * (np - 1);
  return Y >= hw - E ? 1 : (Y <= -(hw - E) ? 2 : 0);
}

__device__ __forceinline__ float sector_alpha(int phys) {
  return ((float)(phys % 18) + 0.5f) * (20.f * 3.14159265358979f / 180.f);
}

// Zeta bin of Z (u): bins of bin_w from Z = -2560 (the smallest Z a cluster can
// have), clamped to the bins of a virtual sector.
__device__ __forceinline__ int zbin(const XsWork& X, long long z) {
  const long long b = (z + 2560) / X.bin_w;
  return (int)(b < 0 ? 0 : (b >= X.n_zb ? X.n_zb - 1 : b));
}

__global__ void k_xs_ends(DevGeom G, DevWork W, XsWork X) {
  const unsigned long long nt = n_tracks_x(W);
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < nt;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const int n = W.trk_ncl[t];
    const int off = W.trk_off[t];
    const int4 pi = W.trk_xyz[off], po = W.trk_xyz[off + n - 1];
    const int ri = (__ldg(reinterpret_cast<const uint4*>(W.clusters) + pi.w).z >> 24) & 0xff;
    const int ro = (__ldg(reinterpret_cast<const uint4*>(W.clusters) + po.w).z >> 24) & 0xff;
    X.side[t] = (uint8_t)(side_code(po.y, G.npads[ro], X.edge_u) | (side_code(pi.y, G.npads[ri], X.edge_u) << 2));
    X.row_in[t] = ri;
    X.row_out[t] = ro;
    X.z_in[t] = pi.z;
    X.z_out[t] = po.z;
    if (((X.side[t] >> 2) & 3) && !W.tracks[t].flags) {   // an entering piece: into its zeta bin
      const int sec = (int)(__ldg(reinterpret_cast<const uint4*>(W.clusters) + pi.w).w >> 24);
      const int vs = vsector_of(G, W, (unsigned)W.trk_first[t], sec);
      atomicAdd(reinterpret_cast<unsigned long long*>(X.bin_off) + (size_t)vs * X.n_zb + zbin(X, pi.z), 1ull);
    }
    X.best_b[t] = ~0ull;
    X.best_a[t] = ~0ull;
    X.link[t] = -1;
    X.prev[t] = -1;
  }
}

// State + covariance (dense) of a fitted track record.
__device__ __forceinline__ void load_fit(const tpc_track& tr, float* s, float (&C)[5][5]) {
#pragma unroll
  for (int i = 0; i < 5; i++) s[i] = tr.par[i];
  int m = 0;
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j <= i; j++) { C[i][j] = tr.cov[m]; C[j][i] = tr.cov[m]; m++; }
}

// Rotation of a state at x by delta (see the header comment); fills the
// nonzero off-identity entries of R.  false if |snp| would reach 0.999.
struct Rot { float r00, r10, r20, r22; };
__device__ __forceinline__ bool rotate_state(float kfac, float* s, float& x, float delta, Rot& R) {
  float sd, cd;
  sincosf(delta, &sd, &cd);
  const float sn = s[2];
  if (fabsf(sn) >= 0.999f) return false;
  const float cs = sqrtf(1.f - sn * sn);
  const float sn2 = sn * cd + cs * sd;
  if (fabsf(sn2) >= 0.999f) return false;
  const float cs2 = sqrtf(1.f - sn2 * sn2);
  R.r00 = cd + (sn2 / cs2) * sd;
  R.r10 = (s[3] / cs2) * sd;
  R.r20 = kfac * s[4] * sd;
  R.r22 = cd - sd * sn / cs;
  const float xn = x * cd - s[0] * sd;
  const float yn = x * sd + s[0] * cd;
  s[0] = yn;
  s[2] = sn2;
  x = xn;
  return true;
}

// Matching chi2 of A (inner piece: state sa, covariance CA at xa in frame
// alpha_a) and B (outer piece); -1 if B cannot be carried to A's reference.
// Early exit: for the symmetric positive definite M = C_A + J C_B J^T,
// d^T M^-1 d >= d_i^2 / M_ii for every i (the minimum of the quadratic form
// over the other components), so a pair with d_i^2 > 4 cut M_ii for i = y or
// zeta has chi2 > cut by a factor far beyond FP32 rounding and is returned as
// +inf without the full 5x5 transform and solve; every other pair gets the
// full chi2, so the accepted pairs and their chi2 are those of the plain
// computation.
__device__ float xs_chi2(float kfac, const float* sa, const float (&CA)[5][5], float xa, float alpha_a,
                         const float (&fb)[24], float cut) {
  // fb: B's tpc_track words par[0..4], x, alpha, chi2, cov[0..14]
  float sb[5], CB[5][5];
#pragma unroll
  for (int i = 0; i < 5; i++) sb[i] = fb[i];
  {
    int m = 0;
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
      for (int j = 0; j <= i; j++) { CB[i][j] = fb[8 + m]; CB[j][i] = fb[8 + m]; m++; }
  }
  float x = fb[5];
  Rot R;
  if (!rotate_state(kfac, sb, x, fb[6] - alpha_a, R)) return -1.f;
  Jac<float> F;
  if (!transport(kfac, sb, xa - x, F)) return -1.f;
  // J = F R: F unit upper triangular with a = F02, b = F04, e = F12, g = F13,
  // h = F14, m = F24; R identity except r00, r10, r20, r22
  float J[5][5];
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j < 5; j++) J[i][j] = (i == j) ? 1.f : 0.f;
  J[0][0] = R.r00 + F.a * R.r20;
  J[0][2] = F.a * R.r22;
  J[0][3] = 0.f;
  J[0][4] = F.b;
  J[1][0] = R.r10 + F.e * R.r20;
  J[1][2] = F.e * R.r22;
  J[1][3] = F.g;
  J[1][4] = F.h;
  J[2][0] = R.r20;
  J[2][2] = R.r22;
  J[2][4] = F.m;
  float d[5];
#pragma unroll
  for (int i = 0; i < 5; i++) d[i] = sa[i] - sb[i];
  // the y and zeta diagonal entries of M first
#pragma unroll
  for (int i = 0; i < 2; i++) {
    float mii = CA[i][i];
#pragma unroll
    for (int k = 0; k < 5; k++)
#pragma unroll
      for (int l = 0; l < 5; l++) mii += J[i][k] * CB[k][l] * J[i][l];
    if (d[i] * d[i] > 4.f * cut * mii) return __int_as_float(0x7f800000);
  }
  // C = C_A + J C_B J^T
  float T[5][5], M[5][5];
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j < 5; j++) {
      float acc = 0.f;
#pragma unroll
      for (int l = 0; l < 5; l++) acc += J[i][l] * CB[l][j];
      T[i][j] = acc;
    }
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j < 5; j++) {
      float acc = 0.f;
#pragma unroll
      for (int l = 0; l < 5; l++) acc += T[i][l] * J[j][l];
      M[i][j] = CA[i][j] + acc;
    }
  return chi2_spd(M, d);
}

// The entering unflagged pieces into their bins (bin_off holds the exclusive
// offsets), each with its candidate-gate fields and fitted state beside it, so
// that the search reads them in bin order; the order within a bin is free:
// the matching keys carry indices.
__global__ void k_xs_fill(DevGeom G, DevWork W, XsWork X) {
  const unsigned long long nt = n_tracks_x(W);
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < nt;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    if (!((X.side[t] >> 2) & 3) || W.tracks[t].flags) continue;
    const int c = W.trk_first[t];
    const int sec = (int)(__ldg(reinterpret_cast<const uint4*>(W.clusters) + c).w >> 24);
    const size_t bin = (size_t)vsector_of(G, W, (unsigned)c, sec) * X.n_zb + zbin(X, X.z_in[t]);
    const unsigned long long e = X.bin_off[bin] + atomicAdd(&X.bin_cur[bin], 1u);
    X.ent[e] = make_uint4((uint32_t)t, (uint32_t)X.z_in[t],
                          (uint32_t)X.row_in[t] | ((uint32_t)((X.side[t] >> 2) & 3) << 8), 0u);
    const uint4* src = reinterpret_cast<const uint4*>(W.tracks + t);
#pragma unroll
    for (int q = 0; q < 6; q++) X.ent_fit[e * 6 + q] = src[q];
  }
}

// One warp per exiting piece A; its lanes share A's candidates, whose chi2 (a
// 5x5 transport, similarity transform and Cholesky solve each) dominates the
// step.  The keys (chi2 bits, index) are unique, so the minima do not depend
// on which lane finds them.
__global__ void k_xs_pairs(DevGeom G, DevParams P, DevWork W, XsWork X) {
  const unsigned long long nt = n_tracks_x(W);
  const int lane = threadIdx.x & 31;
  const unsigned long long wpb = blockDim.x >> 5;
  for (unsigned long long a = blockIdx.x * wpb + (threadIdx.x >> 5); a < nt; a += (unsigned long long)gridDim.x * wpb) {
    const int ex = X.side[a] & 3;
    if (!ex) continue;
    const tpc_track A = W.tracks[a];
    if (A.flags) continue;
    float sa[5], CA[5][5];
    load_fit(A, sa, CA);
    const int c0 = W.trk_first[a];
    const int vs = vsector_of(G, W, (unsigned)c0, A.sector);
    const int phys = vs % G.n_phys, base = vs - phys;
    const int side_base = phys < 18 ? 0 : 18;
    const int nphys = side_base + ((phys - side_base) + (ex == 1 ? 1 : 17)) % 18;
    if (nphys >= G.n_phys) continue;
    const int vb = base + nphys;
    const int want_entry = ex == 1 ? 2 : 1;
    const int ro = X.row_out[a];
    const long long za = X.z_out[a];
    unsigned long long best = ~0ull;
    // the entering unflagged pieces of the neighbouring sector in the zeta
    // bins that can hold |Z_B - Z_A| <= dz (bins are at least dz wide: <= 3)
    const size_t bb = (size_t)vb * X.n_zb;
    const int zl = zbin(X, za - X.dz_u), zh = zbin(X, za + X.dz_u);
    const unsigned long long e1 = X.bin_off[bb + zh + 1];
    unsigned long long e = X.bin_off[bb + zl] + lane;
    uint4 key = e < e1 ? X.ent[e] : make_uint4(0u, 0u, 0u, 0u);
    for (; e < e1; e += 32) {
      const uint4 cur = key;                       // the next candidate's gate fields in flight
      if (e + 32 < e1) key = X.ent[e + 32];
      const unsigned b = cur.x;
      if ((int)(cur.z >> 8) != want_entry || (int)(cur.z & 0xffu) <= ro) continue;
      const long long dz = (long long)(int)cur.y - za;
      if (dz > X.dz_u || dz < -(long long)X.dz_u) continue;
      float fb[24];
#pragma unroll
      for (int q = 0; q < 6; q++) {
        const uint4 v = X.ent_fit[e * 6 + q];
        fb[4 * q] = __uint_as_float(v.x);
        fb[4 * q + 1] = __uint_as_float(v.y);
        fb[4 * q + 2] = __uint_as_float(v.z);
        fb[4 * q + 3] = __uint_as_float(v.w);
      }
      const float c2 = xs_chi2(P.kfac, sa, CA, A.x, A.alpha, fb, X.chi2_cut);
      if (!(c2 >= 0.f) || c2 > X.chi2_cut) continue;
      const unsigned long long cb = (unsigned long long)__float_as_uint(c2) << 32;
      best = min(best, cb | b);
      atomicMin(&X.best_a[b], cb | (unsigned)a);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) X.best_b[a] = best;
  }
}

__global__ void k_xs_link(DevWork W, XsWork X) {
  const unsigned long long nt = n_tracks_x(W);
  unsigned nl = 0;
  for (unsigned long long a = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; a < nt;
       a += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long key = X.best_b[a];
    if (key == ~0ull) continue;
    const unsigned b = (unsigned)key;
    if ((unsigned)X.best_a[b] == (unsigned)a) {
      X.link[a] = (int)b;
      X.prev[b] = (int)a;
      nl++;
    }
  }
  nl = __reduce_add_sync(0xffffffffu, nl);
  if ((threadIdx.x & 31) == 0 && nl) atomicAdd(&X.ctl[1], (unsigned long long)nl);
}

__global__ void k_xs_roots(DevWork W, XsWork X) {
  const unsigned long long nt = n_tracks_x(W);
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < nt;
       t += (unsigned long long)gridDim.x * blockDim.x)
    X.scan[t] = X.prev[t] < 0 ? 1ull : 0ull;
}

// Point i of a chain walk: the piece's cluster list entry and frame.
struct XsPoint { float x, y, z; int sector_phys; };

__device__ __forceinline__ XsPoint xs_point(const DevGeom& G, const DevWork& W, int piece, int l, int Z0) {
  const int4 p = W.trk_xyz[W.trk_off[piece] + l];
  XsPoint q;
  q.x = (float)p.x * kU;
  q.y = (float)p.y * kU;
  q.z = (float)(p.z - Z0) * kU;
  q.sector_phys = (int)(__ldg(reinterpret_cast<const uint4*>(W.clusters) + p.w).w >> 24);
  return q;
}

// U D U^T <- R U D U^T R^T for the sparse rotation Jacobian, by W = R U and a
// modified weighted Gram-Schmidt re-triangularisation (D-weighted rows,
// last to first).
__device__ __forceinline__ void ud_rotate(UD<float>& M, const Rot& R) {
  float w[5][5];
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j < 5; j++) w[i][j] = (i == j) ? 1.f : (j > i ? M.u[i][j] : 0.f);
#pragma unroll
  for (int j = 0; j < 5; j++) {
    const float u0 = w[0][j], u2 = w[2][j];
    w[1][j] += R.r10 * u0;
    w[2][j] = R.r22 * u2 + R.r20 * u0;
    w[0][j] = R.r00 * u0;
  }
  float d[5];
#pragma unroll
  for (int k = 0; k < 5; k++) d[k] = M.d[k];
#pragma unroll
  for (int j = 4; j >= 0; j--) {
    float dj = 0.f;
#pragma unroll
    for (int k = 0; k < 5; k++) dj += d[k] * w[j][k] * w[j][k];
    M.d[j] = dj;
    const float inv = 1.f / dj;
#pragma unroll
    for (int i = 0; i < j; i++) {
      float uij = 0.f;
#pragma unroll
      for (int k = 0; k < 5; k++) uij += d[k] * w[i][k] * w[j][k];
      uij *= inv;
      M.u[i][j] = uij;
#pragma unroll
      for (int k = 0; k < 5; k++) w[i][k] -= uij * w[j][k];
    }
  }
}

// One (y, zeta) measurement in FP32 with the FP64 redo on a failed PD check.
__device__ __forceinline__ float xs_measure(const DevParams& P, float* s, UD<float>& M, float y, float z,
                                            int& flags, int& nfp64) {
  float s0[5];
  UD<float> M0 = M;
#pragma unroll
  for (int a = 0; a < 5; a++) s0[a] = s[a];
  float dchi = ud_update<float, 0>(s, M, y, P.sy2);
  dchi += ud_update<float, 1>(s, M, z, P.sz2);
  if (!ud_pd(M)) {
    double sd[5];
    UD<double> Md;
#pragma unroll
    for (int a = 0; a < 5; a++) {
      sd[a] = s0[a];
      Md.d[a] = M0.d[a];
#pragma unroll
      for (int b = 0; b < 5; b++) Md.u[a][b] = M0.u[a][b];
    }
    double dd = ud_update<double, 0>(sd, Md, (double)y, P.sy2_d);
    dd += ud_update<double, 1>(sd, Md, (double)z, P.sz2_d);
    if (!ud_pd(Md)) flags |= TPC_TRK_NOT_PD;
#pragma unroll
    for (int a = 0; a < 5; a++) {
      s[a] = (float)sd[a];
      M.d[a] = (float)Md.d[a];
#pragma unroll
      for (int b = 0; b < 5; b++) M.u[a][b] = (float)Md.u[a][b];
    }
    dchi = (float)dd;
    nfp64++;
  }
  return dchi;
}

// One thread per merged track (a root piece): numbering, piece assignment,
// record copy (one piece) or multi-frame refit (several).  The grid covers
// every piece (up to 512 blocks per SM): a refit is a long serial chain, and a
// thread given two would take twice the step's time.
__global__ void k_xs_emit(DevGeom G, DevParams P, DevWork W, XsWork X) {
  const unsigned long long nt = n_tracks_x(W);
  for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < nt;
       r += (unsigned long long)gridDim.x * blockDim.x) {
    if (X.prev[r] >= 0) continue;
    const int g = (int)X.scan[r];
    int npieces = 0, ncl = 0, last = (int)r;
    for (int t = (int)r; t >= 0 && npieces < 64; t = X.link[t]) {
      X.group[t] = g;
      npieces++;
      ncl += W.trk_ncl[t];
      last = t;
    }
    if (npieces == 1) {
      X.tracks_out[g] = W.tracks[r];
      continue;
    }
    // ---- refit over all pieces: points innermost (root, cluster 0) first
    const int Z0 = W.trk_xyz[W.trk_off[r]].z;
    const int mid = (ncl - 1) / 2;
    XsPoint p1 = xs_point(G, W, (int)r, 0, Z0), p3 = xs_point(G, W, last, W.trk_ncl[last] - 1, Z0), p2 = p1;
    {
      int t = (int)r, base = 0;
      while (t >= 0 && base + W.trk_ncl[t] <= mid) { base += W.trk_ncl[t]; t = X.link[t]; }
      if (t >= 0) p2 = xs_point(G, W, t, mid - base, Z0);
    }
    const float a3 = sector_alpha(p3.sector_phys);
    auto in_frame3 = [&](const XsPoint& q, float& xo, float& yo) {
      float sd, cd;
      sincosf(sector_alpha(q.sector_phys) - a3, &sd, &cd);
      xo = q.x * cd - q.y * sd;
      yo = q.x * sd + q.y * cd;
    };
    float x1, y1, x2, y2, x3, y3;
    in_frame3(p1, x1, y1);
    in_frame3(p2, x2, y2);
    in_frame3(p3, x3, y3);
    const float ax = x2 - x1, ay = y2 - y1, cx = x3 - x1, cy = y3 - y1;
    const float bx = cx - ax, by = cy - ay;
    const float la = sqrtf(ax * ax + ay * ay), lb = sqrtf(bx * bx + by * by), lc = sqrtf(cx * cx + cy * cy);
    const float kc = 2.f * (ax * cy - ay * cx) / (la * lb * lc);
    const float hh = fminf(1.f, fmaxf(-1.f, 0.5f * kc * lc));
    const float half = asinf(hh);
    const float phic = atan2f(cy, cx);
    const float klc = kc * lc;
    const float arc = fabsf(klc) < 1e-3f ? lc * (1.f + klc * klc * (1.f / 24.f)) : 2.f * half / kc;
    float s[5] = {y3, p3.z, sinf(phic + half), (p3.z - p1.z) / arc, kc / P.kfac};
    UD<float> M;
    float xcur = p3.x, acur = a3;
    int flags = 0, n_used = 0, nfp64 = 0;
    float chi2 = 0.f;
    for (int pass = 0; pass < P.fit_passes; pass++) {
      ud_reset(M, P.c0);
      chi2 = 0.f;
      n_used = 0;
      const bool inward = (pass & 1) == 0;
      // the chain walk keeps its piece's offset, length and sector, and the
      // next point's load is in flight while the current one is fitted
      int t = inward ? last : (int)r;
      int off = W.trk_off[t], nn = W.trk_ncl[t], sec = W.tracks[t].sector;
      int l = inward ? nn - 1 : 0;
      int4 nxt = W.trk_xyz[off + l];
      int nsec = sec;
      bool more = true;
      for (int jj = 0; jj < ncl && more; jj++) {
        const int4 pq = nxt;
        XsPoint q;
        q.x = (float)pq.x * kU;
        q.y = (float)pq.y * kU;
        q.z = (float)(pq.z - Z0) * kU;
        q.sector_phys = nsec;
        if (inward) {
          if (--l < 0) {
            t = X.prev[t];
            if (t >= 0) { off = W.trk_off[t]; nn = W.trk_ncl[t]; sec = W.tracks[t].sector; l = nn - 1; }
          }
        } else {
          if (++l >= nn) {
            t = X.link[t];
            if (t >= 0) { off = W.trk_off[t]; nn = W.trk_ncl[t]; sec = W.tracks[t].sector; l = 0; }
          }
        }
        more = t >= 0;
        if (more) { nxt = W.trk_xyz[off + l]; nsec = sec; }
        const float aq = sector_alpha(q.sector_phys);
        if (aq != acur) {
          Rot Rr;
          if (!rotate_state(P.kfac, s, xcur, acur - aq, Rr)) { flags |= TPC_TRK_STOPPED; break; }
          ud_rotate(M, Rr);
          acur = aq;
        }
        const float dx = q.x - xcur;
        if (dx != 0.f) {
          Jac<float> J;
          if (!transport(P.kfac, s, dx, J)) { flags |= TPC_TRK_STOPPED; break; }
          ud_propagate(M, J);
          xcur = q.x;
        }
        chi2 += xs_measure(P, s, M, q.y, q.z, flags, nfp64);
        n_used++;
      }
    }
    tpc_track out;
    out.par[0] = s[0];
    out.par[1] = s[1] + (float)Z0 * kU;
    out.par[2] = s[2];
    out.par[3] = s[3];
    out.par[4] = s[4];
    out.x = xcur;
    out.alpha = acur;
    out.chi2 = chi2;
    int m = 0;
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
      for (int j = 0; j <= i; j++) {
        float acc = M.d[i] * (j == i ? 1.f : M.u[j][i]);
#pragma unroll
        for (int k = i + 1; k < 5; k++) acc += M.u[i][k] * M.d[k] * M.u[j][k];
        out.cov[m++] = acc;
      }
    out.ndf = 2 * n_used - 5;
    out.n_clusters = ncl;
    out.first_cluster = W.trk_first[r];
    out.sector = W.tracks[r].sector;
    out.flags = (uint16_t)(flags | TPC_TRK_XSECTOR);
    out.n_fp64 = nfp64;
    X.tracks_out[g] = out;
  }
}

__global__ void k_xs_map(DevWork W, XsWork X) {
  unsigned long long n = W.ctr[CTR_NCL];
  if (n > W.cap_cl) n = W.cap_cl;
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < n;
       c += (unsigned long long)gridDim.x * blockDim.x) {
    const int t = W.cl2trk[c];
    X.cl2trk_out[c] = t >= 0 ? X.group[t] : -1;
  }
}

cudaError_t launch_scan(uint64_t* v, const unsigned long long* n_ptr, unsigned long long cap,
                        unsigned long long* state, unsigned int* ticket, unsigned long long* total, uint32_t* err,
                        int n_sm, cudaStream_t st);

static inline unsigned grid_x(unsigned long long cap, int n_sm, int per_sm) {
  unsigned long long g = (cap + 255) / 256;
  const unsigned long long m = (unsigned long long)n_sm * per_sm;
  if (g > m) g = m;
  return (unsigned)(g ? g : 1);
}

cudaError_t launch_xsec(const DevGeom& G, const DevParams& P, const DevWork& W, const XsWork& X, int n_sm,
                        cudaStream_t st) {
  const unsigned g = grid_x(W.cap_ch, n_sm, 8);
  k_xs_ends<<<g, 256, 0, st>>>(G, W, X);
  // bins: counts -> exclusive offsets (n_bins + 1 entries, the last the total)
  cudaError_t e0 = launch_scan(X.bin_off, X.ctl + 3, (unsigned long long)G.n_sectors * X.n_zb + 1, X.bin_state,
                               reinterpret_cast<unsigned int*>(X.ctl + 4), X.ctl + 5, W.err, n_sm, st);
  if (e0 != cudaSuccess) return e0;
  k_xs_fill<<<g, 256, 0, st>>>(G, W, X);
  {   // a warp per piece: 8 pieces per 256-thread block
    unsigned long long gp = (W.cap_ch + 7) / 8;
    const unsigned long long mp = (unsigned long long)n_sm * 16;
    if (gp > mp) gp = mp;
    k_xs_pairs<<<(unsigned)(gp ? gp : 1), 256, 0, st>>>(G, P, W, X);
  }
  k_xs_link<<<g, 256, 0, st>>>(W, X);
  k_xs_roots<<<g, 256, 0, st>>>(W, X);
  cudaError_t e = launch_scan(X.scan, W.ctr + CTR_NTRK, W.cap_ch, X.scan_state,
                              reinterpret_cast<unsigned int*>(X.ctl + 2), X.ctl, W.err, n_sm, st);
  if (e != cudaSuccess) return e;
  {   // a thread per piece up to 148 x 512 x 64 = 4.8 M pieces, so that no thread
      // refits two chains one after the other
    unsigned long long ge = (W.cap_ch + 63) / 64;
    const unsigned long long me = (unsigned long long)n_sm * 512;
    if (ge > me) ge = me;
    k_xs_emit<<<(unsigned)(ge ? ge : 1), 64, 0, st>>>(G, P, W, X);
  }
  k_xs_map<<<grid_x(W.cap_cl, n_sm, 8), 256, 0, st>>>(W, X);
  return cudaGetLastError();
}

}  // namespace tpc
