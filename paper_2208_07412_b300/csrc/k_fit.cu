// k_fit.cu — Kalman-filter helix fit of every track (step 8 of the library's
// definition; the paper's section "Hardware and data flow" says the EPN GPUs
// run the full TPC tracking, whose final stage this is).
//
// One thread per track, the 5-parameter state and its covariance in FP32
// registers.  Exact helix transport (chord form), analytic Jacobian, (y, zeta)
// measurement updates C' = C - K H C then symmetrised.  An update whose result
// fails the positive-definiteness check is recomputed in FP64 from the
// pre-update state and counted; FP64 is used nowhere else.  Measurements are
// integer coordinates relative to the track's first cluster, so they reach
// FP32 exactly before the single scaling to cm.
#include "tpc_internal.cuh"

namespace tpc {

constexpr float kU = 7.8125e-4f;   // cm per u
constexpr double kUd = 7.8125e-4;

template <typename T>
struct Jac { T a, b, e, g, h, m; };  // F02, F04, F12, F13, F14, F24

__device__ __forceinline__ float sgnf(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

// Exact helix transport by dx (state in place).  false: |snp| would reach 0.999.
__device__ __forceinline__ bool transport(float kfac, float* s, float dx, Jac<float>& J) {
  const float k = kfac * s[4];
  const float s1 = s[2], s2 = fmaf(k, dx, s1);
  if (fabsf(s1) >= 0.999f || fabsf(s2) >= 0.999f) return false;
  const float c1 = sqrtf(1.f - s1 * s1), c2 = sqrtf(1.f - s2 * s2);
  const float cc = c1 + c2;
  const float f = (s1 + s2) / cc;
  const float dy = dx * f;
  const float rt = sqrtf(1.f + f * f);
  const float d = fabsf(dx) * rt;
  const float kd = k * d;
  float A;
  if (fabsf(kd) < 1e-3f) {
    A = d * (1.f + kd * kd * (1.f / 24.f));
  } else {
    const float hh = fminf(1.f, fmaxf(-1.f, 0.5f * kd));
    A = 2.f * asinf(hh) / k;
  }
  const float sg = sgnf(dx);
  // Jacobian
  const float fs1 = (1.f + f * (s1 / c1)) / cc;
  const float fs2 = (1.f + f * (s2 / c2)) / cc;
  const float ds2dq = kfac * dx;
  J.a = dx * (fs1 + fs2);
  J.b = dx * fs2 * ds2dq;
  J.m = ds2dq;
  const float x = 0.5f * kd;
  const float Ad = rsqrtf(1.f - x * x);
  float Ak;
  if (fabsf(x) < 0.1f) {
    const float x2 = x * x;
    Ak = (k * d * d * d * 0.25f) *
         ((1.f / 3.f) + x2 * (0.3f + x2 * ((15.f / 56.f) + x2 * (35.f / 144.f))));
  } else {
    Ak = (2.f / (k * k)) * (x * rsqrtf(1.f - x * x) - asinf(x));
  }
  const float dd_df = fabsf(dx) * f / rt;
  J.e = s[3] * sg * Ad * dd_df * (fs1 + fs2);
  J.g = sg * A;
  J.h = s[3] * sg * (Ad * dd_df * fs2 * ds2dq + Ak * kfac);
  s[0] += dy;
  s[1] = fmaf(s[3] * sg, A, s[1]);
  s[2] = s2;
  return true;
}

// C <- F C F^T for the sparse helix Jacobian (full symmetric 5x5 storage).
template <typename T>
__device__ __forceinline__ void propagate_cov(T C[5][5], const Jac<T>& J) {
  T Tm[5][5];
#pragma unroll
  for (int j = 0; j < 5; j++) {
    Tm[0][j] = C[0][j] + J.a * C[2][j] + J.b * C[4][j];
    Tm[1][j] = C[1][j] + J.e * C[2][j] + J.g * C[3][j] + J.h * C[4][j];
    Tm[2][j] = C[2][j] + J.m * C[4][j];
    Tm[3][j] = C[3][j];
    Tm[4][j] = C[4][j];
  }
#pragma unroll
  for (int i = 0; i < 5; i++) {
    C[i][0] = Tm[i][0] + J.a * Tm[i][2] + J.b * Tm[i][4];
    C[i][1] = Tm[i][1] + J.e * Tm[i][2] + J.g * Tm[i][3] + J.h * Tm[i][4];
    C[i][2] = Tm[i][2] + J.m * Tm[i][4];
    C[i][3] = Tm[i][3];
    C[i][4] = Tm[i][4];
  }
}

// Kalman update with measurement (my, mz); returns the chi2 increment and
// whether the result passed the PD check.
template <typename T>
__device__ __forceinline__ T kf_update(T s[5], T C[5][5], T my, T mz, T sy2, T sz2, bool& pd) {
  const T S00 = C[0][0] + sy2, S01 = C[1][0], S11 = C[1][1] + sz2;
  const T det = S00 * S11 - S01 * S01;
  const T I00 = S11 / det, I01 = -S01 / det, I11 = S00 / det;
  const T r0 = my - s[0], r1 = mz - s[1];
  T K[5][2];
#pragma unroll
  for (int i = 0; i < 5; i++) {
    K[i][0] = C[i][0] * I00 + C[i][1] * I01;
    K[i][1] = C[i][0] * I01 + C[i][1] * I11;
  }
#pragma unroll
  for (int i = 0; i < 5; i++) s[i] += K[i][0] * r0 + K[i][1] * r1;
  T N[5][5];
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j < 5; j++) N[i][j] = C[i][j] - (K[i][0] * C[0][j] + K[i][1] * C[1][j]);
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j < 5; j++) C[i][j] = T(0.5) * (N[i][j] + N[j][i]);
#pragma unroll
  for (int i = 0; i < 5; i++) ok = ok && (C[i][i] > T(0));
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = i + 1; j < 5; j++) ok = ok && (C[i][j] * C[i][j] < C[i][i] * C[j][j]);
  pd = ok;
  return r0 * (I00 * r0 + I01 * r1) + r1 * (I01 * r0 + I11 * r1);
}

__global__ void __launch_bounds__(128)
k_fit(DevGeom G, DevParams P, DevWork W) {
  const unsigned long long ntrk = W.ctr[CTR_NTRK];
  const unsigned long long nmax = ntrk < W.cap_ch ? ntrk : W.cap_ch;
  unsigned int fp64_count = 0;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < nmax;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const int n = W.trk_ncl[t];
    const int* lst = W.track_cl + W.trk_off[t];
    const int c0 = lst[0];
    const int X0 = W.cl_x[c0], Y0 = W.cl_y[c0], Z0 = W.cl_z[c0];
    // ---- initial state: circle through innermost, middle and outermost clusters
    const int cm = lst[(n - 1) / 2], co = lst[n - 1];
    const float ax = (float)(W.cl_x[cm] - X0) * kU, ay = (float)(W.cl_y[cm] - Y0) * kU;
    const float cx = (float)(W.cl_x[co] - X0) * kU, cy = (float)(W.cl_y[co] - Y0) * kU;
    const float bx = cx - ax, by = cy - ay;
    const float la = sqrtf(ax * ax + ay * ay), lb = sqrtf(bx * bx + by * by), lc = sqrtf(cx * cx + cy * cy);
    const float kc = 2.f * (ax * cy - ay * cx) / (la * lb * lc);
    const float hh = fminf(1.f, fmaxf(-1.f, 0.5f * kc * lc));
    const float half = asinf(hh);
    const float phic = atan2f(cy, cx);
    const float klc = kc * lc;
    const float arc = fabsf(klc) < 1e-3f ? lc * (1.f + klc * klc * (1.f / 24.f)) : 2.f * half / kc;
    const float zo = (float)(W.cl_z[co] - Z0) * kU;
    float s[5] = {cy, zo, sinf(phic + half), zo / arc, kc / P.kfac};
    float C[5][5];
    int xcur = W.cl_x[co];
    int flags = 0, n_used = 0, nfp64 = 0;
    float chi2 = 0.f;
    for (int pass = 0; pass < P.fit_passes; pass++) {
#pragma unroll
      for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j < 5; j++) C[i][j] = (i == j) ? P.c0[i] : 0.f;
      chi2 = 0.f;
      n_used = 0;
      const bool inward = (pass & 1) == 0;
      for (int jj = 0; jj < n; jj++) {
        const int i = inward ? n - 1 - jj : jj;
        const int c = lst[i];
        const int Xi = W.cl_x[c];
        if (Xi != xcur) {
          Jac<float> J;
          if (!transport(P.kfac, s, (float)(Xi - xcur) * kU, J)) { flags |= TPC_TRK_STOPPED; break; }
          propagate_cov(C, J);
          xcur = Xi;
        }
        const float my = (float)(W.cl_y[c] - Y0) * kU, mz = (float)(W.cl_z[c] - Z0) * kU;
        float s0[5], C0[5][5];
#pragma unroll
        for (int a = 0; a < 5; a++) {
          s0[a] = s[a];
#pragma unroll
          for (int b = 0; b < 5; b++) C0[a][b] = C[a][b];
        }
        bool pd;
        float dchi = kf_update<float>(s, C, my, mz, P.sy2, P.sz2, pd);
        if (!pd) {
          // redo this update in FP64 from the pre-update state
          double sd[5], Cd[5][5];
#pragma unroll
          for (int a = 0; a < 5; a++) {
            sd[a] = s0[a];
#pragma unroll
            for (int b = 0; b < 5; b++) Cd[a][b] = C0[a][b];
          }
          bool pdd;
          double dd = kf_update<double>(sd, Cd, (double)(W.cl_y[c] - Y0) * kUd, (double)(W.cl_z[c] - Z0) * kUd,
                                        P.sy2_d, P.sz2_d, pdd);
#pragma unroll
          for (int a = 0; a < 5; a++) {
            s[a] = (float)sd[a];
#pragma unroll
            for (int b = 0; b < 5; b++) C[a][b] = (float)Cd[a][b];
          }
          dchi = (float)dd;
          if (!pdd) flags |= TPC_TRK_NOT_PD;
          nfp64++;
        }
        chi2 += dchi;
        n_used++;
      }
    }
    // ---- emit
    tpc_track out;
    out.par[0] = s[0] + (float)Y0 * kU;
    out.par[1] = s[1] + (float)Z0 * kU;
    out.par[2] = s[2];
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
      for (int j = 0; j <= i; j++) out.cov[m++] = C[i][j];
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

cudaError_t launch_fit(const DevGeom& G, const DevParams& P, const DevWork& W, int n_sm, cudaStream_t st,
                       int* launches) {
  unsigned long long g = (W.cap_ch + 127) / 128;
  unsigned long long m = (unsigned long long)n_sm * 16;
  if (g > m) g = m;
  k_fit<<<(unsigned)(g ? g : 1), 128, 0, st>>>(G, P, W);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace tpc
