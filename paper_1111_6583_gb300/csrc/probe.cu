// probe.cu -- FMA throughput probe: the measured denominator of the ALU
// rooflines that the benchmark reports for the FP64-bound kernels (and the
// FP32 forms); and a self-test of the bulk-copy barrier wait that the staged
// 1D kernels use (a copy that completes, a wait that must give up).  Not part
// of the method.
#include <cuda_runtime.h>

#include <string>

#include "async_copy.cuh"
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
// SM cycles and global-timer nanoseconds that block 0 spent in its loop: their
// ratio is the SM clock the probe ran at
__device__ unsigned long long g_probe_clk[2];

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x) * T(1e-3) + T(k);
  const bool rec = blockIdx.x == 0 && threadIdx.x == 0;
  long long c0 = 0;
  unsigned long long t0 = 0;
  if (rec) {
    c0 = clock64();
    t0 = claw::global_ns();
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (rec) {
    const long long c1 = clock64();  // after the chains' results are used
    const unsigned long long t1 = claw::global_ns();
    g_probe_clk[0] = (unsigned long long)(c1 - c0) + (s == T(-1234.5) ? 1ull : 0ull);
    g_probe_clk[1] = t1 - t0;
  }
  if (s == T(-1234.5)) g_probe_sink<T> = s;
}

template <typename T>
cudaError_t run_probe(cudaStream_t st, int iters, double* tflops, double* sm_mhz) {
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
  double mhz = 0.0;
  for (int rep = 0; rep < 8 && e == cudaSuccess; ++rep) {  // the first two runs warm up
    cudaEventRecord(a, st);
    fma_probe_kernel<T><<<blocks, kThreads, 0, st>>>(iters, mul, add);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    unsigned long long clk[2] = {0ull, 0ull};
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(clk, g_probe_clk, sizeof(clk));
    if (e == cudaSuccess && rep > 1 && (best == 0.f || ms < best)) {
      best = ms;
      mhz = clk[1] > 0 ? 1e3 * (double)clk[0] / (double)clk[1] : 0.0;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return e;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (sm_mhz) *sm_mhz = mhz;
  return cudaSuccess;
}

// --- bounded barrier waits ------------------------------------------------
constexpr int kProbeWords = 64;  // 256 bytes
__device__ __align__(16) unsigned g_copy_src[kProbeWords];
__device__ unsigned g_copy_dst[kProbeWords];
__device__ unsigned long long g_wait_out[3];  // gave up, copied, ns waited

__device__ __forceinline__ unsigned probe_word(int i) { return 2654435761u * (unsigned)(i + 1); }

__global__ void copy_src_fill_kernel() {
  if (threadIdx.x < kProbeWords) g_copy_src[threadIdx.x] = probe_word(threadIdx.x);
}

// one thread: (1) a barrier that nothing arrives at, waited on for limit_ns:
// the wait must give up; (2) a 256-byte bulk copy into shared memory that
// completes on a second barrier, compared word by word
__global__ void wait_probe_kernel(unsigned long long limit_ns) {
  __shared__ __align__(16) unsigned buf[kProbeWords];
  __shared__ __align__(8) unsigned long long bars[2];
  const unsigned b0 = claw::smem_u32(&bars[0]), b1 = claw::smem_u32(&bars[1]);
  claw::mbar_init(b0, 1u);
  claw::mbar_init(b1, 1u);
  claw::fence_mbar_init();
  const unsigned long long t0 = claw::global_ns();
  const bool got0 = claw::mbar_wait_bounded(b0, 0u, limit_ns);
  const unsigned long long waited = claw::global_ns() - t0;
  claw::fence_proxy_async_smem();
  claw::mbar_arrive_expect_tx(b1, sizeof(buf));
  claw::bulk_g2s(claw::smem_u32(buf), g_copy_src, sizeof(buf), b1);
  bool same = claw::mbar_wait_bounded(b1, 0u);
  if (same) {
    for (int i = 0; i < kProbeWords; ++i) {
      g_copy_dst[i] = buf[i];
      same = same && buf[i] == probe_word(i);
    }
  }
  g_wait_out[0] = got0 ? 0ull : 1ull;
  g_wait_out[1] = same ? 1ull : 0ull;
  g_wait_out[2] = waited;
}

}  // namespace

extern "C" claw_status claw_async_wait_probe(int limit_us, void* stream, int* gave_up,
                                             int* copied, double* waited_us) {
  if (!gave_up || !copied || !waited_us || limit_us < 1 || limit_us > 1000000) {
    claw::set_last_error("claw_async_wait_probe: limit_us in 1..1e6 and non-null outputs");
    return CLAW_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long out[3] = {0ull, 0ull, 0ull};
  copy_src_fill_kernel<<<1, kProbeWords, 0, st>>>();
  wait_probe_kernel<<<1, 1, 0, st>>>((unsigned long long)limit_us * 1000ull);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(out, g_wait_out, sizeof(out), 0,
                                                      cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    claw::set_last_error((std::string("claw_async_wait_probe: ") + cudaGetErrorString(e)).c_str());
    return CLAW_ECUDA;
  }
  *gave_up = (int)out[0];
  *copied = (int)out[1];
  *waited_us = (double)out[2] * 1e-3;
  return CLAW_OK;
}

extern "C" claw_status claw_fma_peak(int prec, void* stream, double* tflops, double* sm_mhz) {
  if (!tflops || (prec != CLAW_FP64 && prec != CLAW_FP32)) {
    claw::set_last_error("claw_fma_peak: prec must be CLAW_FP64 or CLAW_FP32, tflops non-null");
    return CLAW_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = prec == CLAW_FP64 ? run_probe<double>(st, 1 << 13, tflops, sm_mhz)
                                    : run_probe<float>(st, 1 << 17, tflops, sm_mhz);
  if (e != cudaSuccess) {
    claw::set_last_error((std::string("claw_fma_peak: ") + cudaGetErrorString(e)).c_str());
    return CLAW_ECUDA;
  }
  return CLAW_OK;
}
