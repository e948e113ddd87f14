// kfp_probe.cu -- FP64 fused multiply-add rate of the device (measurement utility).
//
// The FP64 sweep is bound by the FP64 pipe, not by HBM: its roofline needs the
// device's DFMA rate, which this measures instead of deriving it from unit counts
// and a nominal clock.  Every thread runs CHAINS independent recurrences
// x <- x * a + b for a fixed number of steps (no memory traffic inside the loop);
// the launch is timed with CUDA events on the caller's stream, and the SM clock
// during the run is taken from the ratio of the SM cycle counter to the global
// nanosecond timer in one thread per block.
//   * many warps and several chains per warp: the throughput of the pipe;
//   * one warp per sub-partition and one chain: one DFMA per dependent step, which
//     gives the latency of a dependent DFMA in cycles.
#include "../../include/kfp_swr.h"

#include <cuda_runtime.h>

namespace {

template <int CHAINS>
__global__ void dfma_probe_kernel(int steps, double a, double b, double* __restrict__ sink,
                                  unsigned long long* __restrict__ clk) {
  double x[CHAINS];
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  unsigned long long c0 = 0, t0 = 0;
  if (threadIdx.x == 0) {
    c0 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  }
  for (int it = 0; it < steps; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int j = 0; j < CHAINS; ++j) x[j] = fma(x[j], a, b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) s += x[j];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) {
    unsigned long long t1;
    const unsigned long long c1 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    clk[2 * blockIdx.x + 0] = c1 - c0;
    clk[2 * blockIdx.x + 1] = t1 - t0;
  }
}

template <int CHAINS>
cudaError_t launch(int blocks, int threads, int steps, double* sink, unsigned long long* clk, cudaStream_t st) {
  // a slightly below 1 and b small keep every x bounded and away from subnormals
  dfma_probe_kernel<CHAINS><<<blocks, threads, 0, st>>>(steps, 0.9999999, 1e-7, sink, clk);
  return cudaGetLastError();
}

}  // namespace

extern "C" kfp_status kfp_probe_fp64_rate(int chains, int warps_per_sm, int steps, double* dfma_per_s,
                                          double* sm_mhz, void* cuda_stream) {
  if (!dfma_per_s || (chains != 1 && chains != 2 && chains != 4 && chains != 8) || warps_per_sm < 1 ||
      warps_per_sm > 32 || steps < 1)
    return KFP_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return KFP_ECUDA;
  }
  const int threads = 32 * warps_per_sm, blocks = sms;  // one block per SM
  double* sink = nullptr;
  unsigned long long* clk = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * (size_t)blocks * threads) != cudaSuccess ||
      cudaMalloc(&clk, sizeof(unsigned long long) * 2 * blocks) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(sink);
    return KFP_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto run = [&](int n) -> cudaError_t {
    switch (chains) {
      case 1: return launch<1>(blocks, threads, n, sink, clk, st);
      case 2: return launch<2>(blocks, threads, n, sink, clk, st);
      case 4: return launch<4>(blocks, threads, n, sink, clk, st);
      default: return launch<8>(blocks, threads, n, sink, clk, st);
    }
  };
  if (e == cudaSuccess) e = run(steps / 10 + 1);  // warm-up (clocks up, code loaded)
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = run(steps);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  unsigned long long c[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(c, clk, sizeof(c), cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(clk);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return KFP_ECUDA;
  }
  const double total = (double)blocks * threads * (double)steps * 8.0 * chains;
  *dfma_per_s = total / (ms * 1e-3);
  if (sm_mhz) *sm_mhz = c[1] > 0 ? 1e3 * (double)c[0] / (double)c[1] : 0.0;
  return KFP_OK;
}
