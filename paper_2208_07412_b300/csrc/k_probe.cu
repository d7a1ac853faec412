// k_probe.cu — FP32 FMA throughput probe: the measured ALU peak against which
// the step-8 fit's achieved FLOP/s is reported (a diagnostics call; the paper
// has no counterpart).
#include <string>

#include "tpc_internal.cuh"

namespace tpc {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;    // independent FMA chains per thread
constexpr int kProbeUnroll = 16;   // FMAs per chain per loop iteration

// Every thread runs kProbeChains independent FMA chains (enough in flight per
// scheduler to hide the FMA latency at 8 blocks of 256 threads per SM) and
// stores their sum, so that no chain can be dropped.
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(float* out, int iters, float a, float b) {
  float x[kProbeChains];
#pragma unroll
  for (int i = 0; i < kProbeChains; i++) x[i] = (float)threadIdx.x * 1e-3f + (float)i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int k = 0; k < kProbeUnroll; k++)
#pragma unroll
      for (int i = 0; i < kProbeChains; i++) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kProbeChains; i++) s += x[i];
  out[blockIdx.x * (unsigned)blockDim.x + threadIdx.x] = s;
}

}  // namespace tpc

using namespace tpc;

extern "C" tpc_status tpc_measure_fma_peak(int device, int reps, double* flops_per_s) {
  auto fail = [](tpc_status st, const std::string& msg) { set_last_error(msg.c_str()); return st; };
  if (!flops_per_s || reps < 1 || reps > 1000) return fail(TPC_E_INVAL, "tpc_measure_fma_peak: bad argument");
  *flops_per_s = 0.0;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(TPC_E_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  int n_sm = 0;
  e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return fail(TPC_E_CUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
  const unsigned grid = (unsigned)n_sm * 8;
  const int iters = 4096;
  float* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double best = 0.0;
  e = cudaMalloc(&out, sizeof(float) * grid * kProbeThreads);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_fma_probe<<<grid, kProbeThreads, 0, st>>>(out, iters, 0.9999999f, 1e-7f);   // warm-up
    e = cudaGetLastError();
  }
  for (int r = 0; r < reps && e == cudaSuccess; r++) {
    cudaEventRecord(e0, st);
    k_fma_probe<<<grid, kProbeThreads, 0, st>>>(out, iters, 0.9999999f, 1e-7f);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms > 0.f) {
      const double flops = 2.0 * kProbeChains * kProbeUnroll * (double)iters * grid * kProbeThreads;
      best = std::max(best, flops / (ms * 1e-3));
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return fail(TPC_E_CUDA, std::string("fma probe: ") + cudaGetErrorString(e));
  *flops_per_s = best;
  return TPC_OK;
}
