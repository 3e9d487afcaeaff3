// probe.cu -- FMA throughput probe: the measured denominator of the ALU
// rooflines that the benchmark reports for the FP64-bound kernels (and the
// FP32 forms).  Not part of the method.
#include <cuda_runtime.h>

#include <string>

#include "clawgpu.h"
#include "kernels.h"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread
constexpr int kThreads = 256;

// Each thread runs kChains independent chains a <- a * b + c for `iters`
// rounds: 2 kChains iters FLOPs per thread.  With b = 1 - 2^-20 and a small c
// the values stay positive and bounded; the sum is stored (to a device
// variable of this file) only if it equals a value it cannot take, which
// keeps every chain live without a store per thread.
template <typename T>
__device__ T g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x) * T(1e-3) + T(k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == T(-1234.5)) g_probe_sink<T> = s;
}

template <typename T>
cudaError_t run_probe(cudaStream_t st, int iters, double* tflops) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<T>, kThreads, 0);
  if (e != cudaSuccess) return e;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  cudaEvent_t a, b;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&b)) != cudaSuccess) {
    cudaEventDestroy(a);
    return e;
  }
  const T mul = T(1) - T(1.0 / 1048576.0), add = T(1e-6);
  float best = 0.f;
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {  // the first run warms up
    cudaEventRecord(a, st);
    fma_probe_kernel<T><<<blocks, kThreads, 0, st>>>(iters, mul, add);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return e;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return cudaSuccess;
}

}  // namespace

extern "C" claw_status claw_fma_peak(int prec, void* stream, double* tflops) {
  if (!tflops || (prec != CLAW_FP64 && prec != CLAW_FP32)) {
    claw::set_last_error("claw_fma_peak: prec must be CLAW_FP64 or CLAW_FP32, tflops non-null");
    return CLAW_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = prec == CLAW_FP64 ? run_probe<double>(st, 1 << 11, tflops)
                                    : run_probe<float>(st, 1 << 15, tflops);
  if (e != cudaSuccess) {
    claw::set_last_error((std::string("claw_fma_peak: ") + cudaGetErrorString(e)).c_str());
    return CLAW_ECUDA;
  }
  return CLAW_OK;
}
