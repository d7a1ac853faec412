// k_fit.cu — Kalman-filter helix fit of every track (step 8 of the library's
// definition; the paper's section "Hardware and data flow" says the EPN GPUs
// run the full TPC tracking, whose final stage this is).
//
// One thread per track, the 5-parameter state and its covariance in FP32
// registers.  Exact helix transport (chord form), analytic Jacobian, (y, zeta)
// measurement updates.  The covariance is kept as U D U^T factors (below): the
// same Kalman filter in exact arithmetic, far less rounding loss in FP32.  An
// update whose result fails the positive-definiteness check (a D entry not
// positive) is recomputed in FP64 from the pre-update state and counted; FP64
// is used nowhere else.  Measurements are
// integer coordinates relative to the track's first cluster, so they reach
// FP32 exactly before the single scaling to cm.
#include "tpc_internal.cuh"

namespace tpc {

constexpr float kU = 7.8125e-4f;   // cm per u
constexpr double kUd = 7.8125e-4;

template <typename T>
struct Jac { T a, b, e, g, h, m; };  // F02, F04, F12, F13, F14, F24

__device__ __forceinline__ float sgnf(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// Exact helix transport by dx (state in place).  false: |snp| would reach
// 0.999.  Written for a short dependency chain: square roots come with their
// reciprocals, and divisions are reciprocals computed off the critical path.
__device__ __forceinline__ bool transport(float kfac, float* s, float dx, Jac<float>& J) {
  const float k = kfac * s[4];
  const float s1 = s[2], s2 = fmaf(k, dx, s1);
  if (fabsf(s1) >= 0.999f || fabsf(s2) >= 0.999f) return false;
  const float e1 = 1.f - s1 * s1, e2 = 1.f - s2 * s2;
  const float rc1 = rsqrtf(e1), rc2 = rsqrtf(e2);     // 1 / cos
  const float c1 = e1 * rc1, c2 = e2 * rc2;
  const float icc = rcp(c1 + c2);
  const float f = (s1 + s2) * icc;
  const float dy = dx * f;
  const float g2 = 1.f + f * f;
  const float irt = rsqrtf(g2);
  const float rt = g2 * irt;
  const float d = fabsf(dx) * rt;
  const float kd = k * d;
  const float x = 0.5f * kd;
  float A, Ak;
  if (fabsf(kd) < 1e-3f) {
    A = d * (1.f + kd * kd * (1.f / 24.f));
  } else {
    A = 2.f * asinf(fminf(1.f, fmaxf(-1.f, x))) * rcp(k);
  }
  const float Ad = rsqrtf(1.f - x * x);
  if (fabsf(x) < 0.1f) {
    const float x2 = x * x;
    Ak = (k * d * d * d * 0.25f) *
         ((1.f / 3.f) + x2 * (0.3f + x2 * ((15.f / 56.f) + x2 * (35.f / 144.f))));
  } else {
    const float ik = rcp(k);
    Ak = 2.f * ik * ik * (x * Ad - asinf(x));
  }
  const float sg = sgnf(dx);
  // Jacobian
  const float fs1 = (1.f + f * s1 * rc1) * icc;
  const float fs2 = (1.f + f * s2 * rc2) * icc;
  const float ds2dq = kfac * dx;
  J.a = dx * (fs1 + fs2);
  J.b = dx * fs2 * ds2dq;
  J.m = ds2dq;
  const float dd_df = fabsf(dx) * f * irt;
  J.e = s[3] * sg * Ad * dd_df * (fs1 + fs2);
  J.g = sg * A;
  J.h = s[3] * sg * (Ad * dd_df * fs2 * ds2dq + Ak * kfac);
  s[0] += dy;
  s[1] = fmaf(s[3] * sg, A, s[1]);
  s[2] = s2;
  return true;
}

// The covariance is carried in factored form C = U D U^T (U unit upper
// triangular, D diagonal).  Exact arithmetic gives the same C as the plain
// update C' = C - K H C; in FP32 the factored form keeps the information that
// the plain form loses to cancellation once C is highly correlated (the
// classical argument for square-root filters).  With the state ordered (y,
// zeta, snp, tgl, q/pT) the helix Jacobian F is unit upper triangular, so the
// time update C' = F C F^T is U' = F U with D unchanged: no re-factorisation.
template <typename T>
struct UD {
  T u[5][5];   // only i < j used (unit diagonal implied)
  T d[5];
};

template <typename T>
__device__ __forceinline__ void ud_reset(UD<T>& M, const float* c0) {
#pragma unroll
  for (int i = 0; i < 5; i++) {
    M.d[i] = T(c0[i]);
#pragma unroll
    for (int j = 0; j < 5; j++) M.u[i][j] = T(0);
  }
}

// U <- F U for the sparse unit upper triangular Jacobian.
template <typename T>
__device__ __forceinline__ void ud_propagate(UD<T>& M, const Jac<T>& J) {
  T(&u)[5][5] = M.u;
  // row 0: + a * row2 + b * row4  (row4 of U = e4, row2 = (0,0,1,u23,u24))
  u[0][2] += J.a;
  u[0][3] += J.a * u[2][3];
  u[0][4] += J.a * u[2][4] + J.b;
  // row 1: + e * row2 + g * row3 + h * row4
  u[1][2] += J.e;
  u[1][3] += J.e * u[2][3] + J.g;
  u[1][4] += J.e * u[2][4] + J.g * u[3][4] + J.h;
  // row 2: + m * row4
  u[2][4] += J.m;
}

// Bierman's scalar measurement update of component `row` (0: y, 1: zeta) with
// variance r.  Updates the state and the factors; returns innovation^2 / its
// variance (the chi2 increment).  The partial sums alpha_j form a short FMA
// chain; their reciprocals are then independent of each other.
template <typename T, int ROW>
__device__ __forceinline__ T ud_update(T s[5], UD<T>& M, T z, T r) {
  T f[5], v[5], b[5], al[5], ia[5];
#pragma unroll
  for (int j = 0; j < 5; j++) {
    f[j] = (j < ROW) ? T(0) : (j == ROW ? T(1) : M.u[ROW][j]);
    v[j] = M.d[j] * f[j];
  }
  al[0] = r + v[0] * f[0];
#pragma unroll
  for (int j = 1; j < 5; j++) al[j] = al[j - 1] + v[j] * f[j];
#pragma unroll
  for (int j = 0; j < 5; j++) ia[j] = rcp(al[j]);
  M.d[0] = M.d[0] * r * ia[0];
  b[0] = v[0];
#pragma unroll
  for (int j = 1; j < 5; j++) {
    const T lam = -f[j] * ia[j - 1];
    M.d[j] = M.d[j] * al[j - 1] * ia[j];
#pragma unroll
    for (int i = 0; i < j; i++) {
      const T uo = M.u[i][j];
      M.u[i][j] = uo + lam * b[i];
      b[i] = b[i] + v[j] * uo;
    }
    b[j] = v[j];
  }
  const T innov = z - s[ROW];
  const T g = ia[4] * innov;
#pragma unroll
  for (int i = 0; i < 5; i++) s[i] += b[i] * g;
  return innov * g;
}

template <typename T>
__device__ __forceinline__ bool ud_pd(const UD<T>& M) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 5; i++) ok = ok && (M.d[i] > T(0)) && (M.d[i] < T(1e30));
  return ok;
}

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
    const int X0 = p0.x, Y0 = p0.y, Z0 = p0.z;
    // ---- initial state: circle through innermost, middle and outermost clusters
    const float ax = (float)(pm.x - X0) * kU, ay = (float)(pm.y - Y0) * kU;
    const float cx = (float)(po.x - X0) * kU, cy = (float)(po.y - Y0) * kU;
    const float bx = cx - ax, by = cy - ay;
    const float la = sqrtf(ax * ax + ay * ay), lb = sqrtf(bx * bx + by * by), lc = sqrtf(cx * cx + cy * cy);
    const float kc = 2.f * (ax * cy - ay * cx) / (la * lb * lc);
    const float hh = fminf(1.f, fmaxf(-1.f, 0.5f * kc * lc));
    const float half = asinf(hh);
    const float phic = atan2f(cy, cx);
    const float klc = kc * lc;
    const float arc = fabsf(klc) < 1e-3f ? lc * (1.f + klc * klc * (1.f / 24.f)) : 2.f * half / kc;
    const float zo = (float)(po.z - Z0) * kU;
    float s[5] = {cy, zo, sinf(phic + half), zo / arc, kc / P.kfac};
    UD<float> M;
    int xcur = po.x;
    int flags = 0, n_used = 0, nfp64 = 0;
    float chi2 = 0.f;
    for (int pass = 0; pass < P.fit_passes; pass++) {
      ud_reset(M, P.c0);
      chi2 = 0.f;
      n_used = 0;
      const bool inward = (pass & 1) == 0;
      int4 nxt = pts[inward ? n - 1 : 0];
      for (int jj = 0; jj < n; jj++) {
        const int4 cur = nxt;
        if (jj + 1 < n) nxt = pts[inward ? n - 2 - jj : jj + 1];   // one cluster ahead
        const int Xi = cur.x;
        if (Xi != xcur) {
          Jac<float> J;
          if (!transport(P.kfac, s, (float)(Xi - xcur) * kU, J)) { flags |= TPC_TRK_STOPPED; break; }
          ud_propagate(M, J);
          xcur = Xi;
        }
        const int dY = cur.y - Y0, dZ = cur.z - Z0;
        float s0[5];
        UD<float> M0 = M;
#pragma unroll
        for (int a = 0; a < 5; a++) s0[a] = s[a];
        float dchi = ud_update<float, 0>(s, M, (float)dY * kU, P.sy2);
        dchi += ud_update<float, 1>(s, M, (float)dZ * kU, P.sz2);
        if (!ud_pd(M)) {
          // redo this update in FP64 from the pre-update state
          double sd[5];
          UD<double> Md;
#pragma unroll
          for (int a = 0; a < 5; a++) {
            sd[a] = s0[a];
            Md.d[a] = M0.d[a];
#pragma unroll
            for (int b = 0; b < 5; b++) Md.u[a][b] = M0.u[a][b];
          }
          double dd = ud_update<double, 0>(sd, Md, (double)dY * kUd, P.sy2_d);
          dd += ud_update<double, 1>(sd, Md, (double)dZ * kUd, P.sz2_d);
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
        chi2 += dchi;
        n_used++;
      }
    }
    // ---- emit: C = U D U^T
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
      for (int j = 0; j <= i; j++) {
        float acc = M.d[i] * (j == i ? 1.f : M.u[j][i]);
#pragma unroll
        for (int k = i + 1; k < 5; k++) acc += M.u[i][k] * M.d[k] * M.u[j][k];
        out.cov[m++] = acc;
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
