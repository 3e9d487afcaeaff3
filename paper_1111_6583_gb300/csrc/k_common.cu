// k_common.cu -- solver-independent kernels: first-dt selection, final-time
// setting, forced steps, activity count, conserved totals.
#include "claw_common.cuh"
#include "kernels.h"

namespace claw {

// dt0 = dt_init if given, else cfl_desired / max_d(smax_d / dx_d) (dt_max when
// nothing moves); bounded by dt_max and clipped to land on t_end.
__global__ void dt_init_kernel(DevCtl* ctls, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  DevCtl* c = ctls + k;
  double dt;
  if (c->dt_init > 0.0) {
    dt = c->dt_init;
  } else {
    double rate = 0.0;
    for (int d = 0; d < c->ndim; ++d) {
      const double v = __longlong_as_double((long long)c->smax[d]) / c->dx[d];
      if (v > rate) rate = v;
    }
    dt = rate > 0.0 ? c->cfl_desired / rate : c->dt_max;
  }
  if (dt > c->dt_max) dt = c->dt_max;
  c->final_ = clip_final(c->t, c->t_end, dt);
  c->dt = dt;
  c->smax[0] = 0ull;
  c->smax[1] = 0ull;
  c->smax[2] = 0ull;
  c->bad = 0u;
  c->arrive = 0u;
}

__global__ void set_t_end_kernel(DevCtl* ctls, int n, double t_end, long long max_rel) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  DevCtl* c = ctls + k;
  c->t_end = t_end;
  c->max_steps = max_rel > 0 ? c->steps + max_rel : 0x7fffffffffffffffLL;
  double dt = c->dt;
  c->final_ = clip_final(c->t, t_end, dt);
  c->dt = dt;
  c->done = (c->status != CLAW_OK) || (c->t >= t_end) ? 1 : 0;
}

__global__ void force_dt_kernel(DevCtl* c, double dt) {
  c->dt = dt;
  c->forced = 1;
  c->final_ = 0;
  c->done = c->status != CLAW_OK ? 1 : 0;
}

__global__ void reset_cur_kernel(DevCtl* c) { c->cur = 0; }

__global__ void count_active_kernel(const DevCtl* ctls, int n, int* out) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int mine = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) mine += ctls[k].done ? 0 : 1;
  atomicAdd(&cnt, mine);
  __syncthreads();
  if (threadIdx.x == 0) *out = cnt;
}

// Conserved totals: per-thread Neumaier sums over a grid-stride range of one
// field, combined pairwise in a fixed tree with an exact two-sum, one (s, c)
// pair per block; the host finishes the sum over blocks in block order.
__device__ __forceinline__ void two_sum_add(double& s, double& c, double s2, double c2) {
  const double t = s + s2;
  const double bp = t - s;
  const double e = (s - (t - bp)) + (s2 - bp);
  s = t;
  c = c + c2 + e;
}

template <typename R>
__global__ void __launch_bounds__(kTotalsThreads)
    totals_kernel(const R* __restrict__ q, const R* __restrict__ kappa, long long ncell,
                  double* partials) {
  const R* f = q + (size_t)blockIdx.y * ncell;
  double s = 0.0, c = 0.0;
  for (long long i = (long long)blockIdx.x * kTotalsThreads + threadIdx.x; i < ncell;
       i += (long long)gridDim.x * kTotalsThreads) {
    const double x = kappa ? (double)f[i] * (double)kappa[i] : (double)f[i];
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  __shared__ double ss[kTotalsThreads], cs[kTotalsThreads];
  ss[threadIdx.x] = s;
  cs[threadIdx.x] = c;
  __syncthreads();
  for (int w = kTotalsThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double a = ss[threadIdx.x], b = cs[threadIdx.x];
      two_sum_add(a, b, ss[threadIdx.x + w], cs[threadIdx.x + w]);
      ss[threadIdx.x] = a;
      cs[threadIdx.x] = b;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const size_t o = ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 2;
    partials[o] = ss[0];
    partials[o + 1] = cs[0];
  }
}

__global__ void gather_ctl_kernel(const Member* members, int n, DevCtl* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = *members[k].ctl;
}

__global__ void set_dry_kernel(DevCtl* c, int dry) { c->dry = dry; }

cudaError_t launch_gather_ctl(const Member* members, int n, DevCtl* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  gather_ctl_kernel<<<(n + 127) / 128, 128, 0, st>>>(members, n, out);
  return cudaGetLastError();
}
cudaError_t launch_set_dry(DevCtl* ctl, int dry, cudaStream_t st) {
  set_dry_kernel<<<1, 1, 0, st>>>(ctl, dry);
  return cudaGetLastError();
}

__global__ void set_dry_n_kernel(DevCtl* c, int n, int dry) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) c[k].dry = dry;
}
cudaError_t launch_set_dry_n(DevCtl* ctls, int n, int dry, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  set_dry_n_kernel<<<(n + 127) / 128, 128, 0, st>>>(ctls, n, dry);
  return cudaGetLastError();
}

// Shu-Osher SSP-RK3: Q1 = Q + dt L(Q); Q2 = 3/4 Q + 1/4 (Q1 + dt L(Q1));
// Q3 = 1/3 Q + 2/3 (Q2 + dt L(Q2)).  Slots: Q^n 0, Q1 1, Q2 2, Q3 1.
static const StageOp kRK3[3] = {
    {0, 1, -1, 0, 0, 0, 1.0, 0.0, 1.0, 0.0, 0.0},
    {1, 2, -1, 0, 0, 0, 1.0, 0.75, 0.25, 0.0, 0.0},
    {2, 1, -1, 0, 0, 1, 1.0, 1.0 / 3.0, 2.0 / 3.0, 0.0, 0.0},
};
// Ketcheson's SSP(10,4), low-storage form: q1 = q1 + dt/6 L(q1) five times;
// q2 = q2/25 + 9 q1/25 and q1 = 15 q2 - 5 q1 = 3/5 Q^n + 2/5 q1 (folded into
// stage 5); four more dt/6 steps; q1 = q2 + 3/5 (q1 + dt/6 L(q1)).  Slots:
// Q^n 0, q1 alternating 1/2, q2 3; the new state lands in slot 2.
static const StageOp kSSP104[10] = {
    {0, 1, -1, 0, 0, 0, 1.0 / 6.0, 0.0, 1.0, 0.0, 0.0},
    {1, 2, -1, 0, 0, 0, 1.0 / 6.0, 0.0, 1.0, 0.0, 0.0},
    {2, 1, -1, 0, 0, 0, 1.0 / 6.0, 0.0, 1.0, 0.0, 0.0},
    {1, 2, -1, 0, 0, 0, 1.0 / 6.0, 0.0, 1.0, 0.0, 0.0},
    {2, 3, 1, 0, 0, 0, 1.0 / 6.0, 1.0 / 25.0, 9.0 / 25.0, 3.0 / 5.0, 2.0 / 5.0},
    {1, 2, -1, 0, 0, 0, 1.0 / 6.0, 0.0, 1.0, 0.0, 0.0},
    {2, 1, -1, 0, 0, 0, 1.0 / 6.0, 0.0, 1.0, 0.0, 0.0},
    {1, 2, -1, 0, 0, 0, 1.0 / 6.0, 0.0, 1.0, 0.0, 0.0},
    {2, 1, -1, 0, 0, 0, 1.0 / 6.0, 0.0, 1.0, 0.0, 0.0},
    {1, 2, -1, 3, 0, 1, 1.0 / 6.0, 1.0, 3.0 / 5.0, 0.0, 0.0},
};

int stage_table(int integrator, const StageOp** ops) {
  if (integrator == 1) {
    *ops = kSSP104;
    return 10;
  }
  *ops = kRK3;
  return 3;
}

__global__ void source_mark_kernel(const Member* __restrict__ members, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    DevCtl* c = members[k].ctl;
    c->src_mark = c->steps;
  }
}

size_t faces_work_bytes(int nd, int nx, int ny, int m, int prec) {
  const size_t nf = nd == 1 ? (size_t)nx + 1
                            : (size_t)(nx + 1) * (ny + 2) + (size_t)(ny + 1) * (nx + 2);
  return nf * 7 * (size_t)m * (prec == 0 ? 8 : 4);
}

__global__ void controllers_kernel(const Member* __restrict__ members, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    DevCtl* c = members[k].ctl;
    if (!c->done) run_controller(c);
  }
}

cudaError_t launch_controllers(const Member* members, int n, cudaStream_t st) {
  controllers_kernel<<<(n + 127) / 128, 128, 0, st>>>(members, n);
  return cudaGetLastError();
}

cudaError_t launch_source_mark(const Member* members, int n, cudaStream_t st) {
  source_mark_kernel<<<(n + 127) / 128, 128, 0, st>>>(members, n);
  return cudaGetLastError();
}

cudaError_t launch_dt_init(DevCtl* ctls, int n, cudaStream_t st) {
  dt_init_kernel<<<(n + 127) / 128, 128, 0, st>>>(ctls, n);
  return cudaGetLastError();
}
cudaError_t launch_set_t_end(DevCtl* ctls, int n, double t_end, long long max_rel,
                             cudaStream_t st) {
  set_t_end_kernel<<<(n + 127) / 128, 128, 0, st>>>(ctls, n, t_end, max_rel);
  return cudaGetLastError();
}
cudaError_t launch_force_dt(DevCtl* ctl, double dt, cudaStream_t st) {
  force_dt_kernel<<<1, 1, 0, st>>>(ctl, dt);
  return cudaGetLastError();
}
cudaError_t launch_reset_cur(DevCtl* ctl, cudaStream_t st) {
  reset_cur_kernel<<<1, 1, 0, st>>>(ctl);
  return cudaGetLastError();
}

// Copy the state in buffer slot ctl->cur into slot dst (nothing when they are
// the same slot), so that the host can queue its read of slot dst without
// first reading the control block.
__global__ void select_copy_kernel(const Member* __restrict__ mem, const DevCtl* __restrict__ ctl,
                                   int dst, size_t bytes) {
  const int cur = ctl->cur;
  if (cur == dst) return;
  const unsigned char* src = (const unsigned char*)mem->q[cur];
  unsigned char* out = (unsigned char*)mem->q[dst];
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  if (((((size_t)src) | ((size_t)out) | bytes) & 15) == 0) {
    const uint4* s4 = (const uint4*)src;
    uint4* o4 = (uint4*)out;
    for (size_t i = t; i < bytes / 16; i += stride) o4[i] = s4[i];
  } else {
    for (size_t i = t; i < bytes; i += stride) out[i] = src[i];
  }
}

cudaError_t launch_select_copy(const Member* mem, const DevCtl* ctl, int dst, size_t bytes,
                               cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  select_copy_kernel<<<(sms > 0 ? sms : 1) * 4, 256, 0, st>>>(mem, ctl, dst, bytes);
  return cudaGetLastError();
}
cudaError_t launch_count_active(const DevCtl* ctls, int n, int* out, cudaStream_t st) {
  count_active_kernel<<<1, 256, 0, st>>>(ctls, n, out);
  return cudaGetLastError();
}
cudaError_t launch_totals(const void* q, const void* kappa, int prec, long long ncell, int m,
                          double* partials, int nblocks, cudaStream_t st) {
  dim3 grid(nblocks, m);
  if (prec == 0)
    totals_kernel<double><<<grid, kTotalsThreads, 0, st>>>((const double*)q, (const double*)kappa,
                                                           ncell, partials);
  else
    totals_kernel<float><<<grid, kTotalsThreads, 0, st>>>((const float*)q, (const float*)kappa,
                                                          ncell, partials);
  return cudaGetLastError();
}

}  // namespace claw
