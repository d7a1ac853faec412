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
