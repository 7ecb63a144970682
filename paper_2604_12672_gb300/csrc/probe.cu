// probe.cu -- arithmetic-throughput probes: the measured denominators of the
// ALU rooflines the stage kernels are reported against (FP32 and FP64
// fused multiply-add rates of this GPU at its current clocks).
#include <cuda_runtime.h>

#include "phl.h"
#include "phl_internal.cuh"

namespace {

constexpr int PR_CHAINS = 8;      // independent FMA chains per thread (hides the pipe latency)
constexpr int PR_ITERS = 2048;    // FMAs per chain
constexpr int PR_THREADS = 256;

// Each thread runs PR_CHAINS independent chains x = x * a + b in registers;
// the result is written only if it matches a value it cannot take, so the
// work is not removed and nothing is stored.
template <typename R>
__global__ void __launch_bounds__(PR_THREADS) k_fma(R a, R b, R never, R *sink) {
  R x[PR_CHAINS];
#pragma unroll
  for (int c = 0; c < PR_CHAINS; ++c) x[c] = (R)(threadIdx.x + c) * (R)1e-3;
  for (int it = 0; it < PR_ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  R s = 0;
#pragma unroll
  for (int c = 0; c < PR_CHAINS; ++c) s += x[c];
  if (s == never) sink[0] = s;
}

}  // namespace

extern "C" phl_status phl_probe_alu(int kind, double *tflops, void *stream) {
  using phl::set_error;
  if (!tflops || (kind != 0 && kind != 1)) return (phl_status)set_error(PHL_EINVAL, "phl_probe_alu: bad argument");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * (kind == 0 ? 8 : 4);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {   // the first run is a warm-up; best of the rest
    cudaEventRecord(e0, s);
    if (kind == 0) k_fma<float><<<blocks, PR_THREADS, 0, s>>>(0.9999f, 1e-4f, -1.0f, nullptr);
    else k_fma<double><<<blocks, PR_THREADS, 0, s>>>(0.9999, 1e-4, -1.0, nullptr);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return (phl_status)set_error(PHL_ECUDA, "phl_probe_alu: %s", cudaGetErrorString(e));
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flop = 2.0 * PR_CHAINS * (double)PR_ITERS * PR_THREADS * blocks;
    if (rep > 0 && ms > 0.0f) best = fmax(best, flop / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *tflops = best;
  return PHL_OK;
}
