// claw_common.cuh -- device-side types shared by the kernels of libclawgpu.
//
// Control block, member (grid) descriptors, method constants, ghost-cell index
// remapping (Sec. 4: periodic, reflecting, outflow, inflow ghost cells done
// inside the tile loads, with no separate halo pass), block reductions and the
// on-device CFL controller (Sec. 4: check the Courant number, choose the next
// step).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "clawgpu.h"

namespace claw {

// ---------------------------------------------------------------------------
// Per-grid controller state, resident in device memory.  Kernels read dt/cur
// at their start; the last block of an attempt (for the 1D row kernel, the
// last warp item, or a controller launch after it) runs the controller, which
// writes the next dt/cur.  Stream order makes the update visible to the next
// launch.
// ---------------------------------------------------------------------------
struct DevCtl {
  double t, dt, t_end, dt_max;
  double cfl_desired, cfl_max;
  double nu_last, nu_max_seen, dt_used;
  double dx[3];
  double idx[3];    // 1 / dx
  double lo[3];     // lower corner of the grid (cell centres for source terms)
  double dt_init;   // first dt (<= 0: from the wave speeds of Q^0)
  unsigned long long smax[3];  // bit patterns of max |s| per direction (non-negative)
  long long steps, rejects, max_steps;
  long long src_mark;  // accepted steps whose source step has been applied
  int cur;          // buffer holding Q^n
  int nbuf;         // 2 (classic), 3 (SharpClaw SSP-RK3) or 4 (SharpClaw SSP(10,4))
  int accept_shift; // buffer rotation on acceptance (slot of the new state)
  int retries, max_retries;
  int status;       // CLAW_OK / CLAW_ECFL / CLAW_ENONPHYSICAL
  int done;         // no more work: t reached t_end, max_steps reached, or error
  int final_;       // current dt was clipped to land on t_end
  int forced;       // current dt was forced by the host (no rejection)
  int accepted;     // last attempt accepted
  int ndim;
  int dry;          // timing runs: attempts leave t, dt and cur unchanged
  unsigned int arrive;  // blocks finished in the current attempt
  unsigned int bad;     // bit 1: non-finite value seen in the current attempt;
                        // bit 2: a bounded wait on an asynchronous copy gave up
};

// One grid of a launch.  Single solves use a table of one member.
struct Member {
  void* q[4];        // state buffers (rotation by DevCtl::cur)
  const void* aux;   // cell aux fields or nullptr
  int nx, ny;        // interior cells (ny = 1 in 1D)
  int ntiles;        // blocks of this member per attempt
  int nz;            // 3D: cells in z (1 otherwise)
  DevCtl* ctl;
  void* work3;       // 3D: per-face fluctuation / correction arrays
  void* qpre;        // Strang-split source: Q^n after the first half source
                     // step, which the step reads in place of slot cur; else null
};

// The step's input in slot cur + rel: Q^n, or with a Strang-split source the
// state after the first half source step.
__device__ __forceinline__ const void* step_input(const Member& mb, int cur, int nbuf, int rel) {
  if (rel == 0) return mb.qpre ? mb.qpre : mb.q[cur];
  return mb.q[(cur + rel) % nbuf];
}

// One stage of a SharpClaw Runge-Kutta method.  Buffer slots are relative to
// DevCtl::cur (slot 0 holds Q^n).  With v = Q[in] + g dt L(Q[in]):
//   Q[out] = a0 Q[sa] + a1 v,   and when out2 >= 0:   Q[out2] = b0 Q[sb] + b1 v.
// The stage marked last runs the CFL controller.
struct StageOp {
  int in, out, out2, sa, sb, last;
  double g, a0, a1, b0, b1;
};

// Work item of a batched launch: (member, tile index within the member).
struct Tile {
  int member;
  int tile;
};

// Method constants in the working precision R.
template <typename R>
struct MConsts {
  R p[8];          // user params
  R inflow[8];     // inflow ghost state
  R aco_c, aco_Z, aco_h;  // acoustics: sound speed, impedance, 1/(2 impedance)
  R g;             // shallow water gravity
  R gamma, gm1;    // Euler
  R weno_eps;
  int weno_r;      // SharpClaw: WENO order 2 weno_r - 1 (0 means 3, WENO5)
  int capa;        // aux field holding the capacity kappa, or -1
  int lim, order, transverse, entropy_fix, char_decomp;
  int bc_lo[3], bc_hi[3];
};

// ---------------------------------------------------------------------------
// ghost-cell remap
// ---------------------------------------------------------------------------
// Map index i along a line of n interior cells to the interior cell whose
// value the ghost takes.  flip = 1 for a reflecting wall (normal component
// negated), inflow = 1 for the fixed inflow state.
__device__ __forceinline__ int bc_map(int i, int n, int bclo, int bchi, int& flip, int& inflow) {
  flip = 0;
  inflow = 0;
  if (i < 0) {
    switch (bclo) {
      case CLAW_BC_PERIODIC: return i + n;
      case CLAW_BC_WALL: flip = 1; return -i - 1;
      case CLAW_BC_INFLOW: inflow = 1; return 0;
      default: return 0;
    }
  }
  if (i >= n) {
    switch (bchi) {
      case CLAW_BC_PERIODIC: return i - n;
      case CLAW_BC_WALL: flip = 1; return 2 * n - 1 - i;
      case CLAW_BC_INFLOW: inflow = 1; return n - 1;
      default: return n - 1;
    }
  }
  return i;
}

// Load cell (c, r) of a field-major array q[M][ny][nx] with ghost remap.  In
// 2D the value of a corner ghost is the y-rule applied to the x-rule value of
// the reflected row (x ghosts are defined on interior rows first).
template <int M, typename R>
__device__ __forceinline__ void load_cell(const MConsts<R>& C, const R* __restrict__ q, int nx,
                                          int ny, int c, int r, int wall_x, int wall_y,
                                          R (&out)[M]) {
  int fy, iy, fx, ix;
  const int rr = bc_map(r, ny, C.bc_lo[1], C.bc_hi[1], fy, iy);
  const int cc = bc_map(c, nx, C.bc_lo[0], C.bc_hi[0], fx, ix);
  if (iy) {
#pragma unroll
    for (int k = 0; k < M; ++k) out[k] = C.inflow[k];
    return;
  }
  if (ix) {
#pragma unroll
    for (int k = 0; k < M; ++k) out[k] = C.inflow[k];
  } else {
    const size_t plane = (size_t)nx * ny;
    const size_t off = (size_t)rr * nx + cc;
#pragma unroll
    for (int k = 0; k < M; ++k) out[k] = __ldg(q + k * plane + off);
#pragma unroll
    for (int k = 0; k < M; ++k)
      if (fx && k == wall_x) out[k] = -out[k];
  }
#pragma unroll
  for (int k = 0; k < M; ++k)
    if (fy && k == wall_y) out[k] = -out[k];
}

// The column part of load_cell's remap, for a thread that keeps its column
// while it walks down rows (computed once per tile).
struct ColMap {
  int cc, fx, ix;
};
template <typename R>
__device__ __forceinline__ ColMap col_map(const MConsts<R>& C, int c, int nx) {
  ColMap m;
  m.cc = bc_map(c, nx, C.bc_lo[0], C.bc_hi[0], m.fx, m.ix);
  return m;
}
// load_cell with the column remap given: the same values
template <int M, typename R>
__device__ __forceinline__ void load_cell_col(const MConsts<R>& C, const R* __restrict__ q, int nx,
                                              int ny, const ColMap& cm, int r, int wall_x,
                                              int wall_y, R (&out)[M]) {
  int fy, iy;
  const int rr = bc_map(r, ny, C.bc_lo[1], C.bc_hi[1], fy, iy);
  if (iy) {
#pragma unroll
    for (int k = 0; k < M; ++k) out[k] = C.inflow[k];
    return;
  }
  if (cm.ix) {
#pragma unroll
    for (int k = 0; k < M; ++k) out[k] = C.inflow[k];
  } else {
    const size_t plane = (size_t)nx * ny;
    const size_t off = (size_t)rr * nx + cm.cc;
#pragma unroll
    for (int k = 0; k < M; ++k) out[k] = __ldg(q + k * plane + off);
#pragma unroll
    for (int k = 0; k < M; ++k)
      if (cm.fx && k == wall_x) out[k] = -out[k];
  }
#pragma unroll
  for (int k = 0; k < M; ++k)
    if (fy && k == wall_y) out[k] = -out[k];
}

// aux fields: same index map, no sign flips, inflow treated as extrapolation
template <int MA, typename R>
__device__ __forceinline__ void load_aux(const MConsts<R>& C, const R* __restrict__ a, int nx,
                                         int ny, int c, int r, R (&out)[MA > 0 ? MA : 1]) {
  if (MA == 0) return;
  int fy, iy, fx, ix;
  const int rr = bc_map(r, ny, C.bc_lo[1], C.bc_hi[1], fy, iy);
  const int cc = bc_map(c, nx, C.bc_lo[0], C.bc_hi[0], fx, ix);
  const size_t plane = (size_t)nx * ny;
#pragma unroll
  for (int k = 0; k < MA; ++k) out[k] = __ldg(a + k * plane + (size_t)rr * nx + cc);
}

// one aux field (runtime index) of cell (c, r) with ghost remap
template <typename R>
__device__ __forceinline__ R load_aux_field(const MConsts<R>& C, const R* __restrict__ a, int nx,
                                            int ny, int c, int r, int field) {
  int fy, iy, fx, ix;
  const int rr = bc_map(r, ny, C.bc_lo[1], C.bc_hi[1], fy, iy);
  const int cc = bc_map(c, nx, C.bc_lo[0], C.bc_hi[0], fx, ix);
  return __ldg(a + (size_t)field * nx * ny + (size_t)rr * nx + cc);
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
// max that keeps NaN (a NaN speed must reach the controller); kept in the
// working precision so FP32 kernels do no FP64 work per interface
template <typename T>
__device__ __forceinline__ T nanmax(T a, T b) { return (b <= a) ? a : b; }


__device__ __forceinline__ int clip_final(double t, double t_end, double& dt) {
  if (t + dt >= t_end) {
    dt = t_end - t;
    return 1;
  }
  return 0;
}

// The CFL controller (one thread).  Courant number nu = max_d dt*smax_d/dx_d;
// reject (keep Q^n, shrink dt by cfl_desired/nu) above cfl_max, otherwise
// accept (advance t, rotate buffers); then choose dt_next = dt*cfl_desired/nu,
// bounded by dt_max and clipped to land on t_end.
static __device__ __noinline__ void run_controller(DevCtl* c) {
  if (c->dry) {
    c->smax[0] = 0ull;
    c->smax[1] = 0ull;
    c->smax[2] = 0ull;
    c->bad = 0u;
    __threadfence();
    c->arrive = 0u;
    return;
  }
  const unsigned bad = atomicOr(&c->bad, 0u);
  const double dt = c->dt;
  double nu = dt * __longlong_as_double((long long)atomicOr(&c->smax[0], 0ull)) / c->dx[0];
  for (int d = 1; d < c->ndim; ++d) {
    const double v = dt * __longlong_as_double((long long)atomicOr(&c->smax[d], 0ull)) / c->dx[d];
    nu = (nu >= v || isnan(nu)) ? nu : v;
  }
  c->accepted = 0;
  if (bad || isnan(nu)) {
    // bit 1: a non-finite value; bit 2: a bounded wait gave up
    c->status = (bad & 2u) ? CLAW_ETIMEOUT : CLAW_ENONPHYSICAL;
    c->done = 1;
  } else if (!c->forced && nu > c->cfl_max) {
    c->rejects += 1;
    c->retries += 1;
    if (c->retries > c->max_retries) {
      c->status = CLAW_ECFL;
      c->done = 1;
    } else {
      double nd = dt * c->cfl_desired / nu;
      if (nd > c->dt_max) nd = c->dt_max;
      c->final_ = clip_final(c->t, c->t_end, nd);
      c->dt = nd;
    }
  } else {
    c->accepted = 1;
    c->t = c->final_ ? c->t_end : c->t + dt;
    c->cur = (c->cur + c->accept_shift) % c->nbuf;
    c->steps += 1;
    c->retries = 0;
    c->nu_last = nu;
    if (nu > c->nu_max_seen) c->nu_max_seen = nu;
    c->dt_used = dt;
    c->forced = 0;
    double nd = nu > 0.0 ? dt * c->cfl_desired / nu : c->dt_max;
    if (nd > c->dt_max) nd = c->dt_max;
    c->final_ = clip_final(c->t, c->t_end, nd);
    c->dt = nd;
    if (c->t >= c->t_end || c->steps >= c->max_steps) c->done = 1;
  }
  c->smax[0] = 0ull;
  c->smax[1] = 0ull;
  c->smax[2] = 0ull;
  c->bad = 0u;
  __threadfence();
  c->arrive = 0u;
}

// Reduce two per-thread maxima and a bad flag over the block (in the working
// precision T; one conversion to double at the end), fold them into the
// control block, and let the last block of the member's attempt run the
// controller (when run_ctl).  Called by every thread of the block; blockDim.x
// must be a multiple of 32 and at most 1024.
template <typename T>
static __device__ __forceinline__ void finish_attempt(DevCtl* ctl, T sx, T sy, int bad, int ntiles,
                                                      bool run_ctl, T sz = T(0)) {
  __shared__ T red_x[32], red_y[32], red_z[32];
  __shared__ int red_bad;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) red_bad = 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sx = nanmax(sx, __shfl_xor_sync(0xffffffffu, sx, o));
    sy = nanmax(sy, __shfl_xor_sync(0xffffffffu, sy, o));
    sz = nanmax(sz, __shfl_xor_sync(0xffffffffu, sz, o));
  }
  __syncthreads();
  if (bad) atomicOr(&red_bad, bad);  // bit 1 non-finite, bit 2 a wait gave up
  if (lane == 0) {
    red_x[warp] = sx;
    red_y[warp] = sy;
    red_z[warp] = sz;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    T a = lane < nw ? red_x[lane] : T(0);
    T b = lane < nw ? red_y[lane] : T(0);
    T z = lane < nw ? red_z[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a = nanmax(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = nanmax(b, __shfl_xor_sync(0xffffffffu, b, o));
      z = nanmax(z, __shfl_xor_sync(0xffffffffu, z, o));
    }
    if (lane == 0) {
      const double ad = (double)a, bd = (double)b, zd = (double)z;
      if (ad != 0.0) atomicMax(&ctl->smax[0], (unsigned long long)__double_as_longlong(ad));
      if (bd != 0.0) atomicMax(&ctl->smax[1], (unsigned long long)__double_as_longlong(bd));
      if (zd != 0.0) atomicMax(&ctl->smax[2], (unsigned long long)__double_as_longlong(zd));
      if (red_bad) atomicOr(&ctl->bad, (unsigned)red_bad);
      if (run_ctl) {
        __threadfence();
        const unsigned prev = atomicAdd(&ctl->arrive, 1u);
        if (prev == (unsigned)ntiles - 1u) {
          __threadfence();
          run_controller(ctl);
        }
      }
    }
  }
}

// Fold a per-thread maximum speed (direction 0) and bad flags into the
// control block with one atomic per warp, no block barrier (the caller
// counts the warp's arrival for the controller, or a controller launch
// follows).  Called by every thread of a full warp.
template <typename T>
static __device__ __forceinline__ void fold_warp(DevCtl* ctl, T sx, int bad) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sx = nanmax(sx, __shfl_xor_sync(0xffffffffu, sx, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    const double d = (double)sx;
    if (d != 0.0) atomicMax(&ctl->smax[0], (unsigned long long)__double_as_longlong(d));
    if (bad) atomicOr(&ctl->bad, (unsigned)bad);  // bit 1 non-finite, bit 2 a wait gave up
  }
}

}  // namespace claw
