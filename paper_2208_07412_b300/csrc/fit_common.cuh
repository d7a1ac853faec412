// fit_common.cuh — the Kalman-filter pieces shared by the per-sector fit
// (k_fit.cu), the cross-sector merge and refit (k_xsec.cu) and the looper-leg
// join (k_loop.cu): exact helix transport with its Jacobian, the U D U^T
// covariance factors, Bierman's scalar update and the matching chi2.
#pragma once
#include "tpc_internal.cuh"

namespace tpc {

constexpr float kU = 7.8125e-4f;   // cm per u
constexpr double kUd = 7.8125e-4;

template <typename T>
struct Jac { T a, b, e, g, h, m; };  // F02, F04, F12, F13, F14, F24

__device__ __forceinline__ float sgnf(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

// FP32 reciprocal: the hardware approximation (2 ulp), not the IEEE-rounded
// one, whose correction steps sit on the fit's serial chain (the longest
// track's 3 x 152 updates set the fit's time).
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// s + e = a + b exactly (Knuth's TwoSum, no condition on the magnitudes).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Exact helix transport by dx (state in place).  false: |snp| would reach
// 0.999.  Written for a short dependency chain: square roots come with their
// reciprocals, and divisions are reciprocals computed off the critical path.
// slo (may be null): the low part of snp, carried so that snp = s[2] + *slo
// keeps the row-to-row increments k dx (~1e-4 of snp on stiff tracks) whole
// instead of rounding each to the ulp of snp.
__device__ __forceinline__ bool transport(float kfac, float* s, float dx, Jac<float>& J, float* slo = nullptr) {
  const float k = kfac * s[4];
  const float s1 = s[2];
  float s2, s2lo = 0.f;
  if (slo) two_sum(s1, fmaf(k, dx, *slo), s2, s2lo);
  else s2 = fmaf(k, dx, s1);
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
  if (fabsf(x) < 0.1f) {
    // arc = (2 / k) asin(kd / 2) = d asin(x) / x, x = kd / 2: the Taylor series
    // of asin(x) / x to x^6 (the next term is below 3e-10 here)
    const float x2 = x * x;
    A = d * (1.f + x2 * ((1.f / 6.f) + x2 * ((3.f / 40.f) + x2 * (5.f / 112.f))));
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
  if (slo) *slo = s2lo;
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
// chain; their reciprocals are then independent of each other.  slo (may be
// null): the low part of snp (see transport), to which the snp correction is
// added before the two parts are renormalised.
template <typename T, int ROW>
__device__ __forceinline__ T ud_update(T s[5], UD<T>& M, T z, T r, float* slo = nullptr) {
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
  for (int i = 0; i < 5; i++) {
    if (i == 2 && slo) {
      float hi, lo;
      two_sum((float)s[2], fmaf((float)b[2], (float)g, *slo), hi, lo);
      s[2] = (T)hi;
      *slo = lo;
    } else {
      s[i] += b[i] * g;
    }
  }
  return innov * g;
}

// Positive-definiteness check of the factors (every D entry in (0, 1e30)),
// without short-circuit branches on the update chain.
template <typename T>
__device__ __forceinline__ bool ud_pd(const UD<T>& M) {
  int ok = 1;
#pragma unroll
  for (int i = 0; i < 5; i++) ok &= (int)(M.d[i] > T(0)) & (int)(M.d[i] < T(1e30));
  return ok != 0;
}

// The FP32 check of the step-8 fit: every D entry above its floor dmin (0 by
// default: the plain positivity check) and below 1e30.  A floor above 0 sends
// updates whose factors have shrunk below it to the FP64 redo.
__device__ __forceinline__ bool ud_pd_above(const UD<float>& M, const float* dmin) {
  int ok = 1;
#pragma unroll
  for (int i = 0; i < 5; i++) ok &= (int)(M.d[i] > dmin[i]) & (int)(M.d[i] < 1e30f);
  return ok != 0;
}

// chi2 = d^T M^-1 d for a symmetric positive definite 5x5 M (Cholesky); -1 if not PD.
__device__ __forceinline__ float chi2_spd(float (&M)[5][5], const float* d) {
  float L[5][5];
#pragma unroll
  for (int j = 0; j < 5; j++) {
    float acc = M[j][j];
#pragma unroll
    for (int k = 0; k < j; k++) acc -= L[j][k] * L[j][k];
    if (!(acc > 0.f)) return -1.f;
    L[j][j] = sqrtf(acc);
    const float inv = 1.f / L[j][j];
#pragma unroll
    for (int i = j + 1; i < 5; i++) {
      float a = M[i][j];
#pragma unroll
      for (int k = 0; k < j; k++) a -= L[i][k] * L[j][k];
      L[i][j] = a * inv;
    }
  }
  float w[5], c2 = 0.f;
#pragma unroll
  for (int i = 0; i < 5; i++) {
    float a = d[i];
#pragma unroll
    for (int k = 0; k < i; k++) a -= L[i][k] * w[k];
    w[i] = a / L[i][i];
    c2 += w[i] * w[i];
  }
  return c2;
}

}  // namespace tpc
