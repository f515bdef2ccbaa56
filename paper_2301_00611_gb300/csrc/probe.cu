// FP64 throughput probe: the measured denominator of the FP64 kernels' roofline.
// Each thread runs kChains independent fused multiply-add chains (enough
// independent work to keep the FP64 pipe's latency hidden; the loop is unrolled so
// that its counter costs next to nothing), launched on a grid
// of resident blocks over every SM; the rate is the flop count over the best
// CUDA-event time of several launches.  The paper has no counterpart.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <string>
#include <thread>

#include "dem.h"

namespace dem {
void set_global_error(const std::string &msg);
}

namespace {
constexpr int kChains = 16;
constexpr int kUnroll = 4;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma_chains(long long iters, double seed,
                                                         double *sink) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  const double b = 0.999999999, d = 1e-9;
  for (long long i = 0; i < iters; i += kUnroll) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], b, d);
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678) *sink = s;   // never true: keeps the chains live
}
// bounded wait for an event (DEM_TIMEOUT_S, default 120 s)
cudaError_t bounded_event_wait(cudaEvent_t ev, bool *timed_out) {
  *timed_out = false;
  const char *env = std::getenv("DEM_TIMEOUT_S");
  double lim = env ? std::atof(env) : 120.0;
  if (!(lim > 0)) lim = 120.0;
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e != cudaErrorNotReady) return e;
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > lim) {
      *timed_out = true;
      return cudaSuccess;
    }
    std::this_thread::yield();
  }
}
}  // namespace

extern "C" dem_status dem_measure_fp64_peak(long long iters, int repeats, void *cuda_stream,
                                            double *tflops) {
  if (!tflops || iters < 1 || repeats < 1) {
    dem::set_global_error("bad probe arguments");
    return DEM_ERR_INVALID_ARG;
  }
  *tflops = 0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains, kThreads, 0);
  double *sink = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&sink, sizeof(double), st);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const long long blocks = (long long)nsm * std::max(per_sm, 1);
  iters = (iters + kUnroll - 1) / kUnroll * kUnroll;
  const double flops = 2.0 * kChains * (double)iters * (double)kThreads * (double)blocks;
  double best = 0;
  bool to = false;
  for (int r = 0; r <= repeats && e == cudaSuccess && !to; ++r) {   // launch 0 warms up
    e = cudaEventRecord(e0, st);
    k_fma_chains<<<(unsigned)blocks, kThreads, 0, st>>>(iters, 1.0 + r, sink);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = bounded_event_wait(e1, &to);
    if (to) break;
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms > 0) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  if (sink) cudaFreeAsync(sink, st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (to) {
    dem::set_global_error("FP64 probe: timed out waiting for the GPU");
    return DEM_ERR_TIMEOUT;
  }
  if (e != cudaSuccess) {
    dem::set_global_error(std::string("FP64 probe: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return DEM_ERR_CUDA;
  }
  *tflops = best;
  return DEM_OK;
}
