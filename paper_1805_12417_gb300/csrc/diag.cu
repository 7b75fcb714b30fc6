// Measured FP64 FMA throughput of the current GPU: the denominator of the
// FP64 inner kernels' arithmetic roofline (they are FP64-pipe bound on this
// part, whose FP64 rate is a small fraction of its FP32 rate).
//
// Every thread runs kChains independent multiply-add recurrences
// a <- a * x + y (x slightly below 1, so a stays near y / (1 - x) = 1 and no
// value overflows or turns subnormal) for kTrips trips; the chains are
// independent so the pipe, not the FMA latency, bounds the rate.  The sum of
// each thread's chains is stored, so no FMA is dead code.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "mrcg.h"

namespace mrcg {
namespace {

constexpr int kChains = 8;
constexpr int kTrips = 4096;

__global__ void __launch_bounds__(kThreads) fp64_fma_kernel(double* out, double x, double y) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 1.0 + 1e-3 * j + 1e-9 * threadIdx.x;
  for (int t = 0; t < kTrips; ++t) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  out[blockIdx.x * (size_t)kThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace mrcg

using namespace mrcg;

extern "C" mrcg_status mrcg_fp64_fma_peak(double* tflops, double* ms) {
  if (!tflops) return MRCG_ERR_INVALID;
  int dev = 0, nsm = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MRCG_ERR_CUDA;
  const int grid = nsm * 8;  // 8 resident 256-thread blocks per SM: enough warps to keep the FP64 pipe busy
  double* out = nullptr;
  if (cudaMalloc(&out, (size_t)grid * kThreads * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return MRCG_ERR_OOM;
  }
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mrcg_status st = MRCG_OK;
  std::vector<float> t;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = MRCG_ERR_CUDA;
  } else {
    const double x = 0.999999, y = 1e-6;
    for (int w = 0; w < 3; ++w) fp64_fma_kernel<<<grid, kThreads, 0, s>>>(out, x, y);
    for (int r = 0; r < 7 && st == MRCG_OK; ++r) {
      cudaEventRecord(e0, s);
      fp64_fma_kernel<<<grid, kThreads, 0, s>>>(out, x, y);
      cudaEventRecord(e1, s);
      float dt = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&dt, e0, e1) != cudaSuccess)
        st = MRCG_ERR_CUDA;
      t.push_back(dt);
    }
  }
  if (st == MRCG_OK && !t.empty()) {
    std::sort(t.begin(), t.end());
    const double best_ms = t.front();
    const double flops = 2.0 * kChains * (double)kTrips * grid * kThreads;
    *tflops = flops / (best_ms * 1e-3) / 1e12;
    if (ms) *ms = best_ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  cudaGetLastError();
  return st;
}
