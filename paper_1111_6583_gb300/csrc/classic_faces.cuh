// classic_faces.cuh -- the classic step (Sec. 2, Eq. (fluxdiff), Eq. (lwflux);
// Sec. 2.1 transverse propagation) on a per-face decomposition, for the cases
// the row-walk kernels do not cover: a capacity function kappa (Eq. (conslaw),
// capacity-form differencing) in 1D or 2D, and 2D solvers whose transverse
// split needs the media of the neighbouring cells.
//
// One attempt = a sweep per direction that writes a record per face (y
// faces: a thread per face loads the four cells of the face's limiter
// stencil and solves the three faces; x faces: a warp takes 30 consecutive
// faces of a line, solves each once and passes the neighbours' waves by
// shuffles; then each face is limited and corrected and its two fluctuations
// split transversely), then an update kernel (a thread per cell) that
// gathers the records of the cell's faces and of the faces whose transverse
// pieces reach it, and whose last block runs the controller.
//
// Capacity: a wave's Courant number uses the capacity of the cell it moves
// into; the correction uses dt/dx times the mean of 1/kappa of the face's two
// cells; a transverse piece is scaled by 1/kappa of the cell its fluctuation
// enters; the cell update is divided by the cell's kappa.
#pragma once

#include "riemann.cuh"

namespace claw {

constexpr int kFacesThreads = 256;

// records per face: amdq, apdq, F, B^-a+, B^+a+, B^-a-, B^+a- (M values each);
// x-face (a, row r) at (r + 1) (nx + 1) + a, y-face (row b, column c) at
// b (nx + 2) + c + 1 (rows r and columns c from -1, the ghost lines)
__host__ __device__ inline size_t faces_count(int nd, int nx, int ny, int dir) {
  if (nd == 1) return dir == 0 ? (size_t)nx + 1 : 0;
  return dir == 0 ? (size_t)(nx + 1) * (ny + 2) : (size_t)(ny + 1) * (nx + 2);
}

// x sweep: a warp takes a chunk of 30 consecutive faces of one line (lanes
// 1..30) and solves each of them once, plus the face below the chunk (lane 0)
// and the one above it (lane 31) for the limiter; chunks per line
constexpr int kFacesChunk = 30;
__host__ __device__ inline int faces_x_chunks(int nx) {
  return (nx + 1 + kFacesChunk - 1) / kFacesChunk;
}
// threads of a sweep launch
__host__ __device__ inline size_t faces_sweep_threads(int nd, int nx, int ny, int dir) {
  if (dir == 1) return faces_count(nd, nx, ny, 1);
  return (size_t)32 * faces_x_chunks(nx) * (nd == 2 ? ny + 2 : 1);
}

template <class RP, typename R, int D>
__global__ void __launch_bounds__(kFacesThreads)
    faces_sweep(const Member* __restrict__ members, const MConsts<R> C, int nd, int in_rel) {
  constexpr int M = RP::M, MW = RP::MW, MA = RP::MA, NC = RP::NCTX;
  constexpr int MAS = MA > 0 ? MA : 1;
  using NZ = typename RP::template NZ<D>;
  const Member& mb = members[0];
  DevCtl* ctl = mb.ctl;
  __shared__ int s_done, s_cur, s_nbuf;
  __shared__ R s_dtdn;
  if (threadIdx.x == 0) {
    s_done = ctl->done;
    s_cur = ctl->cur;
    s_nbuf = ctl->nbuf;
    s_dtdn = (R)(ctl->dt / ctl->dx[D]);
  }
  __syncthreads();
  if (s_done) return;
  const int nx = mb.nx, ny = (nd == 2) ? mb.ny : 1;
  const int n = (D == 0) ? nx : ny, nl = (D == 0) ? ny : nx;
  const int lines = (nd == 2) ? nl + 2 : 1;
  const long long nf = (long long)(n + 1) * lines;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // in_rel 0: Q^n; 1: the x-swept state (second sweep of a split step)
  const R* __restrict__ q = (const R*)step_input(mb, s_cur, s_nbuf, in_rel);
  const R* __restrict__ aux = (const R*)mb.aux;
  R smax = R(0);
  // x sweep: warp chunks (the face of lane t is 30 k - 1 + t on its line; a
  // chunk's halo lanes may stand past the grid's last ghost face, where they
  // load the last ghost cells and own nothing); y sweep: a thread per face
  const int lane = threadIdx.x & 31;
  const int cpl = faces_x_chunks(nx);
  const long long gw = id >> 5;
  const bool live = (D == 0) ? gw < (long long)cpl * lines : id < nf;  // warp-uniform for x
  if (live) {
    // x-faces line by line (row r: faces 0..nx), y-faces row of faces by row
    // of faces (face row b: columns -1..nx), so that consecutive threads read
    // neighbouring cells and write neighbouring records in both sweeps
    const int fraw = (D == 0) ? (int)(gw % cpl) * kFacesChunk - 1 + lane : (int)(id / lines);
    const int l = (nd == 2) ? ((D == 0) ? (int)(gw / cpl) : (int)(id % lines)) - 1 : 0;
    const bool own = (D == 0) ? (lane >= 1 && lane <= kFacesChunk && fraw <= n) : true;
    // every load below stays within the ghost layer (f <= n + 1)
    const int f = (D == 0) ? min(fraw, n + 1) : fraw;
    const R dtdn = s_dtdn;
    R cell[4][M], au[4][MAS];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      // x sweep: only the face's own two cells (its neighbours' waves come
      // from the lanes beside it)
      if (D == 0 && (t == 0 || t == 3)) continue;
      const int a = f - 2 + t;
      const int i = (D == 0) ? a : l, j = (D == 0) ? l : a;
      load_cell<M, R>(C, q, nx, ny, i, j, RP::WALL_X, RP::WALL_Y, cell[t]);
      if (MA > 0) load_aux<MA, R>(C, aux, nx, ny, i, j, au[t]);
    }
    // 1/kappa of the face's two cells (one reciprocal each; every capacity
    // scaling below multiplies by them)
    R ikl = R(1), ikr = R(1);
    if (C.capa >= 0) {
      ikl = FM<R>::rcp(
          load_aux_field<R>(C, aux, nx, ny, D == 0 ? f - 1 : l, D == 0 ? l : f - 1, C.capa));
      ikr = FM<R>::rcp(load_aux_field<R>(C, aux, nx, ny, D == 0 ? f : l, D == 0 ? l : f, C.capa));
    }
    R W[3][MW][M], s[3][MW], am[M], ap[M], x[NC], amx[M], apx[M], xx[NC];
    RP::template solve<D>(C, cell[1], cell[2], au[1], au[2], W[1], s[1], am, ap, x);
    if constexpr (D == 0) {
#pragma unroll
      for (int p = 0; p < MW; ++p) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          W[0][p][k] = __shfl_up_sync(0xffffffffu, W[1][p][k], 1);
          W[2][p][k] = __shfl_down_sync(0xffffffffu, W[1][p][k], 1);
        }
      }
    } else {
      RP::template solve<D>(C, cell[0], cell[1], au[0], au[1], W[0], s[0], amx, apx, xx);
      RP::template solve<D>(C, cell[2], cell[3], au[2], au[3], W[2], s[2], amx, apx, xx);
    }
    // Courant number of the interior faces of interior lines
    if (own && l >= 0 && l < ((nd == 2) ? nl : 1)) {
#pragma unroll
      for (int p = 0; p < MW; ++p) {
        const R sp = s[1][p];
        const R a = C.capa < 0 ? (R)fabs(sp)
                               : (gt0(sp) ? sp * ikr : (lt0(sp) ? -sp * ikl : R(0)));
        smax = nanmax(smax, a);
      }
    }
    R F[M];
    if (C.order == 2) {
      R dot[MW], nrm[MW];
#pragma unroll
      for (int p = 0; p < MW; ++p) {
        R dd = R(0), n2 = R(0);
#pragma unroll
        for (int k = 0; k < M; ++k) {
          if (!NZ::f(p, k)) continue;
          const R up = s[1][p] > R(0) ? W[0][p][k] : W[2][p][k];
          dd += up * W[1][p][k];
          n2 += W[1][p][k] * W[1][p][k];
        }
        dot[p] = dd;
        nrm[p] = n2;
      }
      const R dtc = C.capa < 0 ? dtdn : R(0.5) * (dtdn * ikl + dtdn * ikr);
      correction<RP, R, D>(C, W[1], s[1], dot, nrm, dtc, F);
    } else {
#pragma unroll
      for (int k = 0; k < M; ++k) F[k] = R(0);
    }
    // the face's record
    const size_t NF = (size_t)nf;
    R* rec = (R*)mb.work3 + (D == 0 ? 0 : 7 * (size_t)M * faces_count(nd, nx, ny, 0));
    const size_t fi = (D == 0) ? (size_t)(l + (nd == 2 ? 1 : 0)) * (n + 1) + fraw : (size_t)id;
    R bma[M], bpa[M], bmb[M], bpb[M];
#pragma unroll
    for (int k = 0; k < M; ++k) bma[k] = bpa[k] = bmb[k] = bpb[k] = R(0);
    if (nd == 2 && C.transverse) {
      R tp[M], tm[M];
#pragma unroll
      for (int k = 0; k < M; ++k) {
        tp[k] = C.transverse == 2 ? ap[k] - F[k] : ap[k];
        tm[k] = C.transverse == 2 ? am[k] + F[k] : am[k];
      }
      if constexpr (trans_aux_rp<RP>::value) {
        // media of the transverse neighbours of the two cells
        R mr[MAS], pr[MAS], ml[MAS], pl[MAS];
        if (D == 0) {
          load_aux<MA, R>(C, aux, nx, ny, f, l - 1, mr);
          load_aux<MA, R>(C, aux, nx, ny, f, l + 1, pr);
          load_aux<MA, R>(C, aux, nx, ny, f - 1, l - 1, ml);
          load_aux<MA, R>(C, aux, nx, ny, f - 1, l + 1, pl);
        } else {
          load_aux<MA, R>(C, aux, nx, ny, l - 1, f, mr);
          load_aux<MA, R>(C, aux, nx, ny, l + 1, f, pr);
          load_aux<MA, R>(C, aux, nx, ny, l - 1, f - 1, ml);
          load_aux<MA, R>(C, aux, nx, ny, l + 1, f - 1, pl);
        }
        RP::template trans_aux<D>(C, mr, au[2], pr, tp, bma, bpa);
        RP::template trans_aux<D>(C, ml, au[1], pl, tm, bmb, bpb);
      } else {
        RP::template trans<D>(C, x, tp, bma, bpa);
        RP::template trans<D>(C, x, tm, bmb, bpb);
      }
      if (C.capa >= 0) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          bma[k] *= ikr;
          bpa[k] *= ikr;
          bmb[k] *= ikl;
          bpb[k] *= ikl;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < M && own; ++k) {
      rec[(0 * M + k) * NF + fi] = am[k];
      rec[(1 * M + k) * NF + fi] = ap[k];
      rec[(2 * M + k) * NF + fi] = F[k];
      rec[(3 * M + k) * NF + fi] = bma[k];
      rec[(4 * M + k) * NF + fi] = bpa[k];
      rec[(5 * M + k) * NF + fi] = bmb[k];
      rec[(6 * M + k) * NF + fi] = bpb[k];
    }
  }
  finish_attempt<R>(ctl, D == 0 ? smax : R(0), D == 1 ? smax : R(0), 0, 0, false);
}

template <class RP, typename R>
__global__ void __launch_bounds__(kFacesThreads)
    faces_update(const Member* __restrict__ members, const MConsts<R> C, int nd, int sweep) {
  constexpr int M = RP::M;
  const Member& mb = members[0];
  DevCtl* ctl = mb.ctl;
  __shared__ int s_done, s_cur, s_nbuf;
  __shared__ R s_dtd[2];  // dt/dx, dt/dy
  if (threadIdx.x == 0) {
    s_done = ctl->done;
    s_cur = ctl->cur;
    s_nbuf = ctl->nbuf;
    s_dtd[0] = (R)(ctl->dt / ctl->dx[0]);
    s_dtd[1] = nd == 2 ? (R)(ctl->dt / ctl->dx[1]) : R(0);
  }
  __syncthreads();
  if (s_done) return;
  const int nx = mb.nx, ny = (nd == 2) ? mb.ny : 1;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int bad = 0;
  if (id < (long long)nx * ny) {
    const int i = (int)(id % nx), j = (int)(id / nx);
    // sweep 0: the unsplit step (slot 0 -> 1); dimensional splitting
    // (Godunov): 1 the x-faces only (slot 0 -> 1), 2 the y-faces only
    // (slot 1 -> 2), without transverse terms
    const R* __restrict__ q = (const R*)step_input(mb, s_cur, s_nbuf, sweep == 2 ? 1 : 0);
    R* __restrict__ qo = (R*)mb.q[(s_cur + (sweep == 2 ? 2 : 1)) % s_nbuf];
    const R* __restrict__ aux = (const R*)mb.aux;
    const size_t NX = faces_count(nd, nx, ny, 0), NY = faces_count(nd, nx, ny, 1);
    const R* X = (const R*)mb.work3;
    const R* Y = X + 7 * (size_t)M * NX;
    const R dtdx = s_dtd[0], dtdy = s_dtd[1];
    R cx = dtdx, cy = dtdy;
    if (C.capa >= 0) {
      const R ik = FM<R>::rcp(load_aux_field<R>(C, aux, nx, ny, i, j, C.capa));
      cx = dtdx * ik;
      cy = dtdy * ik;
    }
    // x-face (a, row r) and y-face (b, column c) record indices
    auto xf = [&](int a, int r) -> size_t {
      return nd == 2 ? (size_t)(r + 1) * (nx + 1) + a : (size_t)a;
    };
    auto yf = [&](int c, int b) -> size_t { return (size_t)b * (nx + 2) + (c + 1); };
    const size_t plane = (size_t)nx * ny;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      auto XR = [&](int field, size_t f) { return X[(field * M + k) * NX + f]; };
      auto YR = [&](int field, size_t f) { return Y[(field * M + k) * NY + f]; };
      const R qv = q[k * plane + (size_t)j * nx + i];
      R v;
      if (nd == 1) {
        v = qv - cx * (XR(1, xf(i, 0)) + XR(0, xf(i + 1, 0))) -
            cx * (XR(2, xf(i + 1, 0)) - XR(2, xf(i, 0)));
      } else if (sweep == 1) {
        // x-faces only: the y-face records are not written in this sweep
        v = qv - cx * (XR(1, xf(i, j)) + XR(0, xf(i + 1, j))) -
            cx * (XR(2, xf(i + 1, j)) - XR(2, xf(i, j)));
      } else if (sweep == 2) {
        v = qv - cy * (YR(1, yf(i, j)) + YR(0, yf(i, j + 1))) -
            cy * (YR(2, yf(i, j + 1)) - YR(2, yf(i, j)));
      } else {
        // total correction fluxes: normal part and the transverse pieces that
        // reach the face (order of the terms as in the serial definition)
        auto Ft = [&](int a) {
          const R tr = YR(4, yf(a - 1, j)) + YR(3, yf(a, j)) + YR(6, yf(a - 1, j + 1)) +
                       YR(5, yf(a, j + 1));
          return XR(2, xf(a, j)) - R(0.5) * dtdy * tr;
        };
        auto Gt = [&](int b) {
          const R tr = XR(4, xf(i, b - 1)) + XR(3, xf(i, b)) + XR(6, xf(i + 1, b - 1)) +
                       XR(5, xf(i + 1, b));
          return YR(2, yf(i, b)) - R(0.5) * dtdx * tr;
        };
        const R fl = Ft(i), fr = Ft(i + 1), gb = Gt(j), gt = Gt(j + 1);
        v = qv - cx * (XR(1, xf(i, j)) + XR(0, xf(i + 1, j))) -
            cy * (YR(1, yf(i, j)) + YR(0, yf(i, j + 1))) - cx * (fr - fl) - cy * (gt - gb);
      }
      bad |= !isfinite(v);
      qo[k * plane + (size_t)j * nx + i] = v;
    }
  }
  finish_attempt<R>(ctl, R(0), R(0), bad, mb.ntiles, sweep != 1);
}

}  // namespace claw
