// k_fit.cu — Kalman-filter helix fit of every track (step 8 of the library's
// definition; the paper's section "Hardware and data flow" says the EPN GPUs
// run the full TPC tracking, whose final stage this is).
//
// One thread per track, the 5-parameter state and its covariance in FP32
// registers.  Exact helix transport (chord form), analytic Jacobian, (y, zeta)
// measurement updates.  The covariance is kept as U D U^T factors (below): the
// same Kalman filter in exact arithmetic, far less rounding loss in FP32.  An
// update whose result fails the positive-definiteness check (a D entry not
// above its floor) is recomputed in FP64 from the pre-update state and
// counted; FP64 is used nowhere else.  The fit runs in the integer coordinate
// unit u (7.8125 um, 2^-7 mm) rather than in cm: measurements and row
// distances are integers, exact in FP32, and only the emitted record is scaled
// to cm.  y and zeta are carried relative to the current cluster, snp as a
// high and a low part.
#include "fit_common.cuh"

namespace tpc {

constexpr int kAhead = 4;   // clusters loaded ahead of the one being fitted

template <int kThreads>
__global__ void __launch_bounds__(kThreads)
k_fit(DevGeom G, DevParams P, DevWork W) {
  const unsigned long long ntrk = W.ctr[CTR_NTRK];
  const unsigned long long nmax = ntrk < W.cap_ch ? ntrk : W.cap_ch;
  unsigned int fp64_count = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < nmax;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long t = (unsigned long long)W.fit_order[i];   // longest tracks first
    const int n = W.trk_ncl[t];
    const int4* pts = W.trk_xyz + W.trk_off[t];   // (X, Y, Z, cluster), innermost first
    const int4 p0 = pts[0], pm = pts[(n - 1) / 2], po = pts[n - 1];
    const int c0 = p0.w;
    // ---- initial state: circle through innermost, middle and outermost clusters
    // (integer differences in u: exact in FP32)
    const float ax = (float)(pm.x - p0.x), ay = (float)(pm.y - p0.y);
    const float cx = (float)(po.x - p0.x), cy = (float)(po.y - p0.y);
    const float bx = cx - ax, by = cy - ay;
    const float la = sqrtf(ax * ax + ay * ay), lb = sqrtf(bx * bx + by * by), lc = sqrtf(cx * cx + cy * cy);
    const float kc = 2.f * (ax * cy - ay * cx) / (la * lb * lc);   // 1/u
    const float hh = fminf(1.f, fmaxf(-1.f, 0.5f * kc * lc));
    const float half = asinf(hh);
    const float phic = atan2f(cy, cx);
    const float klc = kc * lc;
    const float arc = fabsf(klc) < 1e-3f ? lc * (1.f + klc * klc * (1.f / 24.f)) : 2.f * half / kc;
    const float zo = (float)(po.z - p0.z);
    // State (y - Yr, zeta - Zr, snp, tgl, q/pT) with y, zeta in u, relative to
    // the integer reference (Yr, Zr), which moves to each cluster before its
    // update: the measurement is then exactly 0 and the state's first two
    // components stay of the size of the residuals, so their FP32 rounding is
    // that of a few hundred u, not of the track's whole extent.
    float s[5] = {0.f, 0.f, sinf(phic + half), zo / arc, kc / P.kfac_u};
    float slo = 0.f;   // low part of snp: snp = s[2] + slo
    int Yr = po.y, Zr = po.z;
    UD<float> M;
    int xcur = po.x;
    int flags = 0, n_used = 0, nfp64 = 0;
    float chi2 = 0.f;
    for (int pass = 0; pass < P.fit_passes; pass++) {
      ud_reset(M, P.c0_u);
      chi2 = 0.f;
      n_used = 0;
      const bool inward = (pass & 1) == 0;
      // the next kAhead clusters in flight (an L2 round trip is longer than one update)
      int4 q[kAhead];
#pragma unroll
      for (int a = 0; a < kAhead; a++) q[a] = a < n ? pts[inward ? n - 1 - a : a] : make_int4(0, 0, 0, 0);
      for (int jj = 0; jj < n; jj++) {
        const int4 cur = q[0];
#pragma unroll
        for (int a = 0; a + 1 < kAhead; a++) q[a] = q[a + 1];
        if (jj + kAhead < n) q[kAhead - 1] = pts[inward ? n - 1 - kAhead - jj : jj + kAhead];
        const int Xi = cur.x;
        if (Xi != xcur) {
          Jac<float> J;
          if (!transport(P.kfac_u, s, (float)(Xi - xcur), J, &slo)) { flags |= TPC_TRK_STOPPED; break; }
          ud_propagate(M, J);
          xcur = Xi;
        }
        // reference to this cluster (integer shifts, exact in FP32 below 2^24 u)
        s[0] -= (float)(cur.y - Yr);
        s[1] -= (float)(cur.z - Zr);
        Yr = cur.y;
        Zr = cur.z;
        float s0[5];
        const float slo0 = slo;
        UD<float> M0 = M;
#pragma unroll
        for (int a = 0; a < 5; a++) s0[a] = s[a];
        float dchi = ud_update<float, 0>(s, M, 0.f, P.sy2_u, &slo);
        dchi += ud_update<float, 1>(s, M, 0.f, P.sz2_u, &slo);
        if (!ud_pd_above(M, P.pd_min_u)) {
          // redo this update in FP64 from the pre-update state
          double sd[5];
          UD<double> Md;
#pragma unroll
          for (int a = 0; a < 5; a++) {
            sd[a] = a == 2 ? (double)s0[2] + (double)slo0 : (double)s0[a];
            Md.d[a] = M0.d[a];
#pragma unroll
            for (int b = 0; b < 5; b++) Md.u[a][b] = M0.u[a][b];
          }
          double dd = ud_update<double, 0>(sd, Md, 0.0, P.sy2_ud);
          dd += ud_update<double, 1>(sd, Md, 0.0, P.sz2_ud);
          if (!ud_pd(Md)) flags |= TPC_TRK_NOT_PD;
#pragma unroll
          for (int a = 0; a < 5; a++) {
            s[a] = (float)sd[a];
            if (a == 2) slo = (float)(sd[2] - (double)s[2]);
            M.d[a] = (float)Md.d[a];
#pragma unroll
            for (int b = 0; b < 5; b++) M.u[a][b] = (float)Md.u[a][b];
          }
          dchi = (float)dd;
          nfp64++;
        }
        chi2 += dchi;
        n_used++;
      }
    }
    // ---- emit in cm: C = U D U^T, rows / columns of y and zeta scaled by kU
    tpc_track out;
    out.par[0] = ((float)Yr + s[0]) * kU;
    out.par[1] = (float)Zr * kU + s[1] * kU;
    out.par[2] = s[2] + slo;
    out.par[3] = s[3];
    out.par[4] = s[4];
    out.x = (float)xcur * kU;
    const int sec = (int)(__ldg(reinterpret_cast<const uint4*>(W.clusters) + c0).w >> 24);
    out.alpha = ((float)(sec % 18) + 0.5f) * (20.f * 3.14159265358979f / 180.f);
    out.chi2 = chi2;
    int m = 0;
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
      for (int j = 0; j <= i; j++) {
        float acc = M.d[i] * (j == i ? 1.f : M.u[j][i]);
#pragma unroll
        for (int k = i + 1; k < 5; k++) acc += M.u[i][k] * M.d[k] * M.u[j][k];
        const float sc = (i < 2 ? kU : 1.f) * (j < 2 ? kU : 1.f);
        out.cov[m++] = acc * sc;
      }
    out.ndf = 2 * n_used - 5;
    out.n_clusters = n;
    out.first_cluster = W.trk_first[t];
    out.sector = (int16_t)sec;
    out.flags = (uint16_t)flags;
    out.n_fp64 = nfp64;
    const uint4* src = reinterpret_cast<const uint4*>(&out);
    uint4* dst = reinterpret_cast<uint4*>(W.tracks + t);
#pragma unroll
    for (int q = 0; q < (int)(sizeof(tpc_track) / 16); q++) dst[q] = src[q];
    fp64_count += nfp64;
  }
  if (fp64_count) atomicAdd(&W.ctr[CTR_NFP64], (unsigned long long)fp64_count);
}

cudaError_t launch_fit(const DevGeom& G, const DevParams& P, const DevWork& W, int n_sm, const LaunchCfg& L,
                       cudaStream_t st, int* launches) {
  const int nt = L.fit_threads;
  unsigned long long g = (W.cap_ch + nt - 1) / nt;
  unsigned long long m = (unsigned long long)n_sm * L.fit_blocks_per_sm;
  if (g > m) g = m;
  const unsigned grid = (unsigned)(g ? g : 1);
  if (nt == 32)
    k_fit<32><<<grid, 32, 0, st>>>(G, P, W);
  else if (nt == 128)
    k_fit<128><<<grid, 128, 0, st>>>(G, P, W);
  else
    k_fit<64><<<grid, 64, 0, st>>>(G, P, W);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace tpc
