// FP64 FMA throughput of the GPU: the denominator of the FP64 path's roofline. The paper's cost
// statement (Sec. 2: O(Dcut^15) flops per step) fixes the work; how fast the FP64 squeeze can
// run is set by the rate of the CUDA cores' double-precision FMA units, which these kernels
// measure (independent FMA chains in every thread, enough warps to cover the FMA latency, and
// the 4 x 4 outer-product accumulation of a register-blocked GEMM).
#include <algorithm>

#include "kernels.h"

namespace hotrg {
namespace {

constexpr int kUnroll = 16;   // FMAs per chain per loop iteration

// kChains independent FMA chains per thread
template <int kChains>
__global__ void __launch_bounds__(256) k_dfma_chains(long long iters, double seed, double* sink) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = seed + 1e-9 * threadIdx.x + i;
  // x -> x m + c contracts towards c / (1 - m) and stays finite for any number of iterations
  const double m = 0.999999999999, c = 1e-13;
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  // a store the compiler cannot remove, taken by no thread in practice
  if (s == -1.0) sink[blockIdx.x] = s;
}

// 4 x 4 outer-product accumulation, the inner loop of a register-blocked GEMM: 16 independent
// accumulators fed by 8 operands per iteration (the operands drift slowly so nothing is constant)
__global__ void __launch_bounds__(256) k_dfma_outer(long long iters, double seed, double* sink) {
  double a[4], b[4], acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a[i] = seed + 1e-9 * threadIdx.x + 0.25 * i;
    b[i] = 1.0 - 1e-12 * i;
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  }
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = fma(a[i], -1e-16, a[i]);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s += acc[i][j];
  if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace hotrg

using namespace hotrg;

extern "C" int hotrg_bench_fp64_fma(long long iters, double* sink, double* tflops, void* stream) {
  if (iters < 1 || iters > (1LL << 32) || !sink || !tflops) return HOTRG_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return HOTRG_EDEVICE;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return HOTRG_EDEVICE;
  }
  // 8, 16 and 32 chains per thread (the FMA latency must be covered); the best rate is the peak
  double best = 0.0;
  bool ok = true;
  // flops per thread and loop iteration: chains x kUnroll FMAs, or 8 x (16 + 4) for the outer product
  auto run = [&](auto kernel, int fmas_per_iter) {
    kernel<<<blocks, threads, 0, s>>>(iters, 1.0, sink);  // warm-up (clocks, code load)
    cudaEventRecord(e0, s);
    kernel<<<blocks, threads, 0, s>>>(iters, 1.0, sink);
    cudaEventRecord(e1, s);
    count_launches(2);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) {
      ok = false;
      return;
    }
    const double flops = 2.0 * (double)iters * fmas_per_iter * (double)blocks * threads;
    best = std::max(best, flops / (ms * 1e-3) / 1e12);
  };
  run(k_dfma_chains<8>, 8 * kUnroll);
  if (ok) run(k_dfma_chains<16>, 16 * kUnroll);
  if (ok) run(k_dfma_chains<32>, 32 * kUnroll);
  if (ok) run(k_dfma_outer, 8 * 20);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) {
    cudaGetLastError();
    return HOTRG_EDEVICE;
  }
  *tflops = best;
  return HOTRG_OK;
}
