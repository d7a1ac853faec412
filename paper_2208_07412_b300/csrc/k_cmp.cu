// k_cmp.cu — optional track-model compression of the clusters on tracks
// (step 10 of the library's definition; the paper's section "Hardware and data
// flow" gives the online reconstruction as the means to reduce the TPC data).
//
// Per step-8 track, one thread: the fitted parameters at the innermost cluster
// are carried along the exact helix from row to row (predicted state only);
// each cluster's measured (y, zeta) minus the prediction at its row, divided
// by the step and rounded (ties away from zero), is its pair of 8-bit codes
// when both are within +-127; otherwise, and after a failed transport, the
// cluster is escaped (kept raw).  Decoding adds code * step to the prediction,
// so a coded position is within half a step of the measured one.
#include "fit_common.cuh"

namespace tpc {

__global__ void k_compress(DevParams P, DevWork W, CmpWork C) {
  unsigned long long ntrk = W.ctr[CTR_NTRK];
  if (ntrk > W.cap_ch) ntrk = W.cap_ch;
  unsigned coded = 0, escaped = 0;
  const float iy = 1.f / C.step_y, iz = 1.f / C.step_z;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < ntrk;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const int n = W.trk_ncl[t];
    const int4* pts = W.trk_xyz + W.trk_off[t];   // innermost first
    const tpc_track& tr = W.tracks[t];
    float s[5] = {tr.par[0], tr.par[1], tr.par[2], tr.par[3], tr.par[4]};
    float x = tr.x;
    bool ok = true;
    for (int i = 0; i < n; i++) {
      const int4 p = pts[i];
      const float xc = (float)p.x * kU;
      if (ok && xc != x) {
        Jac<float> J;
        if (transport(P.kfac, s, xc - x, J)) x = xc; else ok = false;
      }
      uint8_t st = 2;
      if (ok) {
        const float cy = roundf(((float)p.y * kU - s[0]) * iy), cz = roundf(((float)p.z * kU - s[1]) * iz);
        if (fabsf(cy) <= 127.f && fabsf(cz) <= 127.f) {
          C.code_y[p.w] = (int8_t)cy;
          C.code_z[p.w] = (int8_t)cz;
          st = 1;
        }
      }
      C.status[p.w] = st;
      if (st == 1) coded++; else escaped++;
    }
  }
  coded = __reduce_add_sync(0xffffffffu, coded);
  escaped = __reduce_add_sync(0xffffffffu, escaped);
  if ((threadIdx.x & 31) == 0) {
    if (coded) atomicAdd(&C.ctl[0], (unsigned long long)coded);
    if (escaped) atomicAdd(&C.ctl[1], (unsigned long long)escaped);
  }
}

cudaError_t launch_compress(const DevParams& P, const DevWork& W, const CmpWork& C, int n_sm, cudaStream_t st) {
  unsigned long long g = (W.cap_ch + 63) / 64;
  const unsigned long long m = (unsigned long long)n_sm * 16;
  if (g > m) g = m;
  k_compress<<<(unsigned)(g ? g : 1), 64, 0, st>>>(P, W, C);
  return cudaGetLastError();
}

}  // namespace tpc

// ---------------------------------------------------------------------------
// Optional drift calibration (step 11 of the library's definition; the paper
// lists calibration among the EPNs' tasks, "Hardware and data flow").  Per
// step-8 track with >= 20 clusters and no flag: its state carried along the
// exact helix to x = 0 (the beam axis), used if |y| < 3 cm there; t_v = zeta /
// (zeta per time bin).  The mode of floor(t_v) over 2^20 bins (lowest bin on
// ties) seeds a mean over |t_v - (b* + 0.5)| <= 3, then one over |t_v - mean|
// <= 1.5.  Sums in FP64 atomics (order-dependent only in the last bits).
namespace tpc {

constexpr int kCalBins = 1 << 20;

__global__ void k_calib_tracks(DevParams P, DevWork W, CalWork C) {
  unsigned long long ntrk = W.ctr[CTR_NTRK];
  if (ntrk > W.cap_ch) ntrk = W.cap_ch;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < ntrk;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const tpc_track& tr = W.tracks[t];
    float tv = -1.f;
    if (tr.n_clusters >= 20 && tr.flags == 0) {
      float s[5] = {tr.par[0], tr.par[1], tr.par[2], tr.par[3], tr.par[4]};
      Jac<float> J;
      if (transport(P.kfac, s, -tr.x, J) && fabsf(s[0]) < 3.f) tv = s[1] / C.zeta_per_bin;
    }
    C.tv[t] = tv;
    if (tv >= 0.f && tv < (float)kCalBins) atomicAdd(&C.hist[(int)floorf(tv)], 1u);
  }
}

// Mode: key = count << 32 | (kCalBins - 1 - bin), maximised (lowest bin on ties).
__global__ void k_calib_mode(CalWork C) {
  unsigned long long best = 0;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < kCalBins; b += gridDim.x * blockDim.x) {
    const unsigned n = C.hist[b];
    if (n) best = max(best, ((unsigned long long)n << 32) | (unsigned)(kCalBins - 1 - b));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0 && best) atomicMax(C.mode, best);
}

__global__ void k_calib_mean(DevWork W, CalWork C, int pass) {
  unsigned long long ntrk = W.ctr[CTR_NTRK];
  if (ntrk > W.cap_ch) ntrk = W.cap_ch;
  double centre, win;
  if (pass == 0) {
    const unsigned long long m = *C.mode;
    if (!m) return;
    centre = (double)(kCalBins - 1 - (int)(unsigned)m) + 0.5;
    win = 3.0;
  } else {
    if (C.cnt[0] == 0) return;
    centre = C.sum[0] / (double)C.cnt[0];
    win = 1.5;
  }
  double s = 0.0;
  unsigned n = 0;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < ntrk;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const float tv = C.tv[t];
    if (tv >= 0.f && fabs((double)tv - centre) <= win) { s += (double)tv; n++; }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    n += __shfl_xor_sync(0xffffffffu, n, o);
  }
  if ((threadIdx.x & 31) == 0 && n) {
    atomicAdd(&C.sum[pass], s);
    atomicAdd(&C.cnt[pass], (unsigned long long)n);
  }
}

cudaError_t launch_calibrate(const DevParams& P, const DevWork& W, const CalWork& C, int n_sm, cudaStream_t st) {
  unsigned long long g = (W.cap_ch + 255) / 256;
  const unsigned long long m = (unsigned long long)n_sm * 8;
  if (g > m) g = m;
  k_calib_tracks<<<(unsigned)(g ? g : 1), 256, 0, st>>>(P, W, C);
  k_calib_mode<<<n_sm * 4, 256, 0, st>>>(C);
  k_calib_mean<<<(unsigned)(g ? g : 1), 256, 0, st>>>(W, C, 0);
  k_calib_mean<<<(unsigned)(g ? g : 1), 256, 0, st>>>(W, C, 1);
  return cudaGetLastError();
}

}  // namespace tpc
