// classic3d.cuh -- 3D unsplit Clawpack-classic step (LeVeque 1997): normal
// solves, limited corrections, transverse and double-transverse propagation,
// for scalar advection and linear acoustics.
//
// One attempt = three face sweeps (one per direction; a zero fill of the
// per-face arrays before them only without transverse terms) and an update
// kernel whose last block runs the controller.
// Transverse pieces: a fluctuation a that enters cell c across a d-face adds
// -dt/(2 dx_d) E^+-a to the e-faces of c; the part E^+-a has moved on into
// cell c +- e, so its third-direction split F^+-E^+-a moves 1/6 (dt/dx_d)
// (dt/dx_e) of flux correction from the f-faces of c to those of c +- e
// (six orderings of the directions give the corner-transport-upwind term).
//
// Every face value is written by one thread, in a fixed order.  y and z
// sweeps: a block owns a square patch of lines along its direction (plus a
// one-line halo it solves again) and walks them together, cell by cell; at
// each cell every line puts the fluctuation entering its cell across the two
// sweep faces, and that sum's transverse splits, into shared memory, and each
// owner line then gathers what its cell's two upper transverse faces receive.
// x sweep: lanes along x, a block of y lines walking z planes
// (classic3d_xsweep below), so that a warp's accesses stay contiguous.
// Results do not depend on scheduling, so batches and servers match single
// solves bit for bit.
#pragma once

#include "kernels.h"
#include "riemann.cuh"

namespace claw {

// cell (i, j, k) of q[M][nz][ny][nx] with ghost remap: x rule, then y rule on
// the x-remapped value, then z rule (corners defined as x, y, z fills in turn)
template <int M, typename R>
__device__ __forceinline__ void load_cell3(const MConsts<R>& C, const R* __restrict__ q, int nx,
                                           int ny, int nz, int i, int j, int k, int wall0,
                                           int wall1, int wall2, R (&out)[M]) {
  int fz, iz, fy, iy, fx, ix;
  const int kk = bc_map(k, nz, C.bc_lo[2], C.bc_hi[2], fz, iz);
  const int jj = bc_map(j, ny, C.bc_lo[1], C.bc_hi[1], fy, iy);
  const int ii = bc_map(i, nx, C.bc_lo[0], C.bc_hi[0], fx, ix);
  if (iz || iy || ix) {
    // an inflow rule at any level replaces the value below it
#pragma unroll
    for (int c = 0; c < M; ++c) out[c] = C.inflow[c];
    if (iz) return;
    if (iy) {
#pragma unroll
      for (int c = 0; c < M; ++c)
        if (fz && c == wall2) out[c] = -out[c];
      return;
    }
  } else {
    const size_t plane = (size_t)nx * ny * nz;
    const size_t off = ((size_t)kk * ny + jj) * nx + ii;
#pragma unroll
    for (int c = 0; c < M; ++c) out[c] = __ldg(q + c * plane + off);
#pragma unroll
    for (int c = 0; c < M; ++c)
      if (fx && c == wall0) out[c] = -out[c];
  }
#pragma unroll
  for (int c = 0; c < M; ++c) {
    if (fy && c == wall1) out[c] = -out[c];
    if (fz && c == wall2) out[c] = -out[c];
  }
}

// 3D transverse split in direction E of a fluctuation a
template <class RP, typename R, int E>
struct Trans3;

template <typename R, int E>
struct Trans3<RpAdvection<R, 3>, R, E> {
  __device__ static __forceinline__ void split(const MConsts<R>& C, const R (&a)[1], R (&em)[1],
                                               R (&ep)[1]) {
    const R v = C.p[E];
    em[0] = fmin(v, R(0)) * a[0];
    ep[0] = fmax(v, R(0)) * a[0];
  }
};

template <typename R, int E>
struct Trans3<RpAcoustics<R, 3>, R, E> {
  __device__ static __forceinline__ void split(const MConsts<R>& C, const R (&a)[4], R (&em)[4],
                                               R (&ep)[4]) {
    constexpr int e = 1 + E;
    const R Z = C.aco_Z, c = C.aco_c, h = C.aco_h;
    const R b1 = (Z * a[e] - a[0]) * h;
    const R b2 = (Z * a[e] + a[0]) * h;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      em[k] = R(0);
      ep[k] = R(0);
    }
    em[0] = c * Z * b1;
    em[e] = -c * b1;
    ep[0] = c * Z * b2;
    ep[e] = c * b2;
  }
};

// per-face arrays: for direction d, faces (nx+[d==0]) x (ny+[d==1]) x (nz+[d==2]),
// each with M values of A^-dQ, A^+dQ and the total correction flux
struct Faces3 {
  size_t n[3];       // faces per direction
  size_t off_am[3], off_ap[3], off_fc[3];  // element offsets into the work array
};

__host__ __device__ inline void faces3_layout(int nx, int ny, int nz, int M, Faces3& f) {
  size_t o = 0;
  for (int d = 0; d < 3; ++d) {
    f.n[d] = (size_t)(nx + (d == 0)) * (ny + (d == 1)) * (nz + (d == 2));
    f.off_am[d] = o;
    o += f.n[d] * M;
    f.off_ap[d] = o;
    o += f.n[d] * M;
    f.off_fc[d] = o;
    o += f.n[d] * M;
  }
}

// the M values of one face record (M consecutive elements of a record whose
// offset is a multiple of M; the face arrays start on 256-byte boundaries):
// one 16-byte access per 16 bytes when M = 4, so a thread's record moves in
// one (FP32) or two (FP64) accesses instead of four
template <int M, typename R>
__device__ __forceinline__ void ld_rec(const R* p, R (&v)[M]) {
  if constexpr (M == 4 && sizeof(R) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (M == 4 && sizeof(R) == 8) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  } else {
#pragma unroll
    for (int c = 0; c < M; ++c) v[c] = p[c];
  }
}

template <int M, typename R>
__device__ __forceinline__ void st_rec(R* p, const R (&v)[M]) {
  if constexpr (M == 4 && sizeof(R) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (M == 4 && sizeof(R) == 8) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  } else {
#pragma unroll
    for (int c = 0; c < M; ++c) p[c] = v[c];
  }
}

template <typename R>
__device__ __forceinline__ size_t face_index(int e, int nx, int ny, const int (&f)[3]) {
  const int NXF = nx + (e == 0), NYF = ny + (e == 1);
  return ((size_t)f[2] * NYF + f[1]) * NXF + f[0];
}

// add v to the correction flux of face f in direction e, which this thread
// alone updates in the current launch (earlier launches' sums are already in
// place by stream order), when the face bounds an interior cell.  The adds
// are reductions done in the L2: with one writer per value and launch the sum
// is the one a read-modify-write gives (FP32 reductions flush a subnormal
// result to zero), and no load sits on the thread's path to the next cell.
template <int M, typename R>
__device__ __forceinline__ void add_fc_own(R* __restrict__ work, const Faces3& L, int e, int nx,
                                           int ny, int nz, const int (&f)[3], const R (&v)[M]) {
  const int n3[3] = {nx, ny, nz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int hi = (d == e) ? n3[d] : n3[d] - 1;
    if (f[d] < 0 || f[d] > hi) return;
  }
  R* base = work + L.off_fc[e] + face_index<R>(e, nx, ny, f) * M;
  if constexpr (M == 4 && sizeof(R) == 4) {
    // one 16-byte vector reduction for the record (16-byte aligned)
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(base), "f"(v[0]),
                 "f"(v[1]), "f"(v[2]), "f"(v[3])
                 : "memory");
  } else {
#pragma unroll
    for (int c = 0; c < M; ++c) atomicAdd(base + c, v[c]);
  }
}

// sweep blocks: kPatch3d x kPatch3d lines (owners: the inner kPatch3d - 2
// squared), kSeg3d cells along the sweep direction
constexpr int kPatch3d = 16;
constexpr int kSeg3d = 32;

__host__ __device__ inline void sweep3d_grid(int D, int nx, int ny, int nz, int& npf, int& nps,
                                             int& nseg) {
  const int n3[3] = {nx, ny, nz};
  const int E1 = (D + 1) % 3, E2 = (D + 2) % 3;
  const int FA = (E2 == 0) ? E2 : E1, SA = (FA == E1) ? E2 : E1;
  constexpr int PO = kPatch3d - 2;
  // owner lines -1 .. n-1 in both transverse directions
  npf = (n3[FA] + 1 + PO - 1) / PO;
  nps = (n3[SA] + 1 + PO - 1) / PO;
  nseg = (n3[D] + kSeg3d - 1) / kSeg3d;
}

template <class RP, typename R, int D>
__global__ void __launch_bounds__(kPatch3d * kPatch3d)
    classic3d_sweep(const Member* __restrict__ members, const MConsts<R> C) {
  constexpr int M = RP::M, MW = RP::MW;
  constexpr int E1 = (D + 1) % 3, E2 = (D + 2) % 3;
  constexpr int P = kPatch3d, PO = P - 2, T = kSeg3d;
  // the transverse direction that runs fastest across threads (x when it is one)
  constexpr int FA = (E2 == 0) ? E2 : E1, SA = (FA == E1) ? E2 : E1;
  // per line: the entering sum S and its splits E1^-, E1^+, E2^-, E2^+
  __shared__ R sh[5][M][P * P];
  const Member& mb = members[0];
  DevCtl* ctl = mb.ctl;
  __shared__ int s_done, s_cur;
  __shared__ R s_k[3];  // dt/dx_d for d = 0, 1, 2
  if (threadIdx.x == 0) {
    s_done = ctl->done;
    s_cur = ctl->cur;
    for (int d = 0; d < 3; ++d) s_k[d] = (R)(ctl->dt / ctl->dx[d]);
  }
  __syncthreads();
  if (s_done) return;
  const int nx = mb.nx, ny = mb.ny, nz = mb.nz;
  const int n3[3] = {nx, ny, nz};
  const int nd = n3[D];
  int npf, nps, nseg;
  sweep3d_grid(D, nx, ny, nz, npf, nps, nseg);
  const int pf = blockIdx.x % npf, ps = (blockIdx.x / npf) % nps, seg = blockIdx.x / (npf * nps);
  const int tf = threadIdx.x % P, ts = threadIdx.x / P;
  int line[3];
  line[D] = 0;
  line[FA] = pf * PO - 2 + tf;
  line[SA] = ps * PO - 2 + ts;
  const bool owner = tf >= 1 && tf <= PO && ts >= 1 && ts <= PO &&
                     line[FA] <= n3[FA] - 1 && line[SA] <= n3[SA] - 1;
  const bool interior_line =
      line[E1] >= 0 && line[E1] < n3[E1] && line[E2] >= 0 && line[E2] < n3[E2];
  const int s0 = seg * T, s1 = min(s0 + T, nd);
  const bool last = s1 == nd;
  const R* __restrict__ q = (const R*)mb.q[s_cur];
  R* __restrict__ work = (R*)mb.work3;
  Faces3 L;
  faces3_layout(nx, ny, nz, M, L);
  const R dtdn = s_k[D];
  const int me = ts * P + tf;
  // shared-memory slot of the line offset by (d1, d2) in (E1, E2)
  auto nb = [&](int d1, int d2) {
    const int df = FA == E1 ? d1 : d2, ds = FA == E1 ? d2 : d1;
    return (ts + ds) * P + (tf + df);
  };
  // lines past the second ghost line (the last patch of a small grid) load
  // that ghost line; no owner reads them
  const int la = min(line[E1], n3[E1] + 1), lb = min(line[E2], n3[E2] + 1);
  auto load = [&](int i, R (&out)[M]) {
    int c3[3];
    c3[D] = i;
    c3[E1] = la;
    c3[E2] = lb;
    load_cell3<M, R>(C, q, nx, ny, nz, c3[0], c3[1], c3[2], RP::WALL_X, 2, 3, out);
  };
  // window: waves of faces i-1 (Wl), i (Wc) and i+1 (Wr); face i lies
  // between cells i-1 and i
  R Wl[MW][M], Wc[MW][M], Wr[MW][M], sl[MW], sc[MW], sr[MW];
  R amc[M], apc[M], amr[M], apr[M];
  R cl[M], cr[M];
  {
    R x[RP::NCTX], amt[M], apt[M];
    load(s0 - 2, cl);
    load(s0 - 1, cr);
    RP::template solve<D>(C, cl, cr, nullptr, nullptr, Wl, sl, amt, apt, x);
    load(s0, cl);
    RP::template solve<D>(C, cr, cl, nullptr, nullptr, Wc, sc, amc, apc, x);
  }
  R smax = R(0);
  R Pv[M];  // A+dQ - F of face i-1 (enters cell i-1 from the left)
#pragma unroll
  for (int c = 0; c < M; ++c) Pv[c] = R(0);
  const R tfF = C.transverse == 2 ? R(1) : R(0);
  // faces s0 .. s1 (face s1 closes cell s1-1; it belongs to the next segment
  // unless this is the last one)
  for (int i = s0; i <= s1; ++i) {
    {
      R x[RP::NCTX];
      load(i + 1, cr);
      RP::template solve<D>(C, cl, cr, nullptr, nullptr, Wr, sr, amr, apr, x);
#pragma unroll
      for (int c = 0; c < M; ++c) cl[c] = cr[c];
    }
    R F[M];
    if (C.order == 2) {
      R dot[MW], nrm[MW];
      constexpr int KS = strength_k<RP, D>();
#pragma unroll
      for (int p = 0; p < MW; ++p) {
        if constexpr (KS >= 0) {
          dot[p] = sc[p] > R(0) ? Wl[p][KS] : Wr[p][KS];
          nrm[p] = Wc[p][KS];
        } else {
          R d_ = R(0), n2 = R(0);
#pragma unroll
          for (int c = 0; c < M; ++c) {
            const R up = sc[p] > R(0) ? Wl[p][c] : Wr[p][c];
            d_ += up * Wc[p][c];
            n2 += Wc[p][c] * Wc[p][c];
          }
          dot[p] = d_;
          nrm[p] = n2;
        }
      }
      correction<RP, R, D>(C, Wc, sc, dot, nrm, dtdn, F);
    } else {
#pragma unroll
      for (int c = 0; c < M; ++c) F[c] = R(0);
    }
    if (owner && interior_line && (i < s1 || last)) {
#pragma unroll
      for (int p = 0; p < MW; ++p) smax = nanmax(smax, (R)fabs(sc[p]));
      int f[3];
      f[D] = i;
      f[E1] = line[E1];
      f[E2] = line[E2];
      const size_t fi = face_index<R>(D, nx, ny, f);
      st_rec<M, R>(work + L.off_am[D] + fi * M, amc);
      st_rec<M, R>(work + L.off_ap[D] + fi * M, apc);
      add_fc_own<M, R>(work, L, D, nx, ny, nz, f, F);
    }
    if (C.transverse) {
      if (i > s0) {
        // cell i-1: A+dQ - F of face i-1 plus A-dQ + F of face i, and its
        // splits in both transverse directions (linear solvers: one sum)
        R S[M], e1m[M], e1p[M], e2m[M], e2p[M];
#pragma unroll
        for (int c = 0; c < M; ++c) S[c] = Pv[c] + (amc[c] + tfF * F[c]);
        Trans3<RP, R, E1>::split(C, S, e1m, e1p);
        Trans3<RP, R, E2>::split(C, S, e2m, e2p);
#pragma unroll
        for (int c = 0; c < M; ++c) {
          sh[0][c][me] = S[c];
          sh[1][c][me] = e1m[c];
          sh[2][c][me] = e1p[c];
          sh[3][c][me] = e2m[c];
          sh[4][c][me] = e2p[c];
        }
      }
#pragma unroll
      for (int c = 0; c < M; ++c) Pv[c] = apc[c] - tfF * F[c];
      __syncthreads();
      if (i > s0 && owner) {
        // the upper g-face of cell X = i-1 (g = E1, then E2), e the third
        // direction: transverse h G^+_g S(X) + h G^-_g S(X+g); double
        // transverse from X and X+g (their own faces) and from X-+e, X+g-+e
        // (pieces that moved on into X, X+g); the splits are linear, so each
        // side's pieces are summed before one split
        const R h = R(-0.5) * dtdn;
#pragma unroll
        for (int gi = 0; gi < 2; ++gi) {
          const int g = gi == 0 ? E1 : E2;
          const int e = gi == 0 ? E2 : E1;
          const int cem = gi == 0 ? 3 : 1, cep = gi == 0 ? 4 : 2;  // e-split slots
          const R k6 = dtdn * s_k[e] * (R(1) / R(6));
          const int d1g = gi == 0 ? 1 : 0, d2g = gi == 0 ? 0 : 1;  // +g in (E1, E2)
          const int d1e = gi == 0 ? 0 : 1, d2e = gi == 0 ? 1 : 0;  // +e in (E1, E2)
          const int x0 = me, xg = nb(d1g, d2g);
          const int xme = nb(-d1e, -d2e), xpe = nb(d1e, d2e);
          const int xgme = nb(d1g - d1e, d2g - d2e), xgpe = nb(d1g + d1e, d2g + d2e);
          R A[M], B[M];
#pragma unroll
          for (int c = 0; c < M; ++c) {
            A[c] = h * sh[0][c][x0] + k6 * (sh[cep][c][x0] - sh[cem][c][x0]) -
                   k6 * (sh[cep][c][xme] - sh[cem][c][xpe]);
            B[c] = h * sh[0][c][xg] + k6 * (sh[cep][c][xg] - sh[cem][c][xg]) -
                   k6 * (sh[cep][c][xgme] - sh[cem][c][xgpe]);
          }
          R am_[M], ap_[M], bm_[M], bp_[M], v[M];
          if (gi == 0) {
            Trans3<RP, R, E1>::split(C, A, am_, ap_);
            Trans3<RP, R, E1>::split(C, B, bm_, bp_);
          } else {
            Trans3<RP, R, E2>::split(C, A, am_, ap_);
            Trans3<RP, R, E2>::split(C, B, bm_, bp_);
          }
#pragma unroll
          for (int c = 0; c < M; ++c) v[c] = ap_[c] + bm_[c];
          int f[3];
          f[D] = i - 1;
          f[g] = line[g] + 1;
          f[e] = line[e];
          add_fc_own<M, R>(work, L, g, nx, ny, nz, f, v);
        }
      }
      __syncthreads();
    }
    // slide the window
#pragma unroll
    for (int p = 0; p < MW; ++p) {
      sl[p] = sc[p];
      sc[p] = sr[p];
#pragma unroll
      for (int c = 0; c < M; ++c) {
        Wl[p][c] = Wc[p][c];
        Wc[p][c] = Wr[p][c];
      }
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
      amc[c] = amr[c];
      apc[c] = apr[c];
    }
  }
  R sx = D == 0 ? smax : R(0), sy = D == 1 ? smax : R(0), sz = D == 2 ? smax : R(0);
  finish_attempt<R>(ctl, sx, sy, 0, 0, false, sz);
}

// The x sweep with lanes along x.  In the walking sweep above, x is the
// sweep direction and the 32 threads of a warp sit on 32 different (y, z)
// lines, so every load and face store of a warp touches 32 separate sectors.
// Here a warp holds 32 consecutive cells of one x line (28 owned cells, two
// halo cells below and two above), the block's NW warps hold NW consecutive
// y lines (the first and last are halo lines), and the block walks the z
// planes of a segment.  Neighbour waves along x come by warp shuffles; what
// crosses lines goes through shared memory once per plane; every global
// access of a warp is one contiguous run along x.
//
// The transverse terms of the walking sweep regroup by line.  For a cell X
// of plane k with entering sum S and its splits (e1 = y, e2 = z):
//   A_y(X) = h S(X) + k6z (e2p(X) - e2m(X)) - k6z (e2p(X - z) - e2m(X + z))
//   A_z(X) = h S(X) + k6y (e1p(X) - e1m(X)) - k6y (e1p(X - y) - e1m(X + y))
// (h = -dt/(2 dx), k6e = (dt/dx)(dt/dx_e)/6).  The upper y-face of X gets
// G_y^+ A_y(X) + G_y^- A_y(X + y) and the upper z-face
// G_z^+ A_z(X) + G_z^- A_z(X + z).  A_y needs only the cell's own line (three
// planes, kept in registers) and A_z the neighbouring lines of the same plane
// (shared memory); A_y of the line above goes through shared memory too and
// A_z of the plane above is the next step's value on the same line.
//
// With transverse terms on, this sweep is the first writer of every record
// of the step: each x-face record, and the correction flux of each y- and
// z-face, gets exactly one owner, which stores it (no zero fill, no
// read-modify-write).  Without transverse terms the y- and z-face fluxes
// stay as the zero fill left them.
constexpr int kXOwn3d = 28;  // owned cells per warp (lanes 2 .. 29)
constexpr int kXSweepLines = 12;  // y lines per block (owners: the inner ten)
constexpr int kZSeg3d = 32;  // owned planes per block

__host__ __device__ inline void xsweep3d_grid(int NW, int nx, int ny, int nz, int& nxc, int& nyb,
                                              int& nzs) {
  nxc = (nx + kXOwn3d - 1) / kXOwn3d;
  nyb = (ny + 1 + (NW - 2) - 1) / (NW - 2);  // owner lines -1 .. ny-1
  nzs = (nz + 1 + kZSeg3d - 1) / kZSeg3d;    // owner planes -1 .. nz-1
}

// NB = 2: the shared exchange is double-buffered by plane parity (one
// barrier per plane); NB = 1: one buffer, a second barrier before it is
// rewritten
template <class RP, typename R, int NW, int NB>
__global__ void __launch_bounds__(32 * NW)
    classic3d_xsweep(const Member* __restrict__ members, const MConsts<R> C) {
  constexpr int M = RP::M, MW = RP::MW;
  static_assert(NW >= 3 && (NB == 1 || NB == 2), "three or more lines, one or two buffers");
  // per buffer: e1m and e1p of plane p, A_y of plane p - 1, per line and lane
  __shared__ R sh[NB][3][M][NW][32];
  const Member& mb = members[0];
  DevCtl* ctl = mb.ctl;
  __shared__ int s_done, s_cur;
  __shared__ R s_k[3];
  if (threadIdx.x == 0) {
    s_done = ctl->done;
    s_cur = ctl->cur;
    for (int d = 0; d < 3; ++d) s_k[d] = (R)(ctl->dt / ctl->dx[d]);
  }
  __syncthreads();
  if (s_done) return;
  const int nx = mb.nx, ny = mb.ny, nz = mb.nz;
  int nxc, nyb, nzs;
  xsweep3d_grid(NW, nx, ny, nz, nxc, nyb, nzs);
  const int bx = blockIdx.x % nxc, by = (blockIdx.x / nxc) % nyb, bz = blockIdx.x / (nxc * nyb);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int x0 = bx * kXOwn3d;
  const int j = by * (NW - 2) - 2 + w;  // this warp's line; owners are warps 1 .. NW-2
  const int z0 = bz * kZSeg3d - 1, z1 = min(z0 + kZSeg3d, nz);  // owner planes [z0, z1)
  // lane l holds cell x0 - 2 + l and the face below it; lines and cells past
  // the second ghost layer load that layer (no owner reads them)
  const int f = x0 - 2 + lane;
  const int xc = min(f, nx + 1), jl = min(j, ny + 1);
  const bool owner_line = w >= 1 && w <= NW - 2 && j <= ny - 1;
  const bool interior_line = j >= 0;  // j <= ny - 1 for owners
  const bool own_cell = lane >= 2 && lane <= 29 && f <= nx - 1;
  const bool own_face = (lane >= 2 && lane <= 29 && f <= nx) || (lane == 30 && f == nx);
  const R* __restrict__ q = (const R*)mb.q[s_cur];
  R* __restrict__ work = (R*)mb.work3;
  Faces3 L;
  faces3_layout(nx, ny, nz, M, L);
  const R dtdn = s_k[0];
  const R tfF = C.transverse == 2 ? R(1) : R(0);
  const R h = R(-0.5) * dtdn;
  const R k6y = dtdn * s_k[1] * (R(1) / R(6)), k6z = dtdn * s_k[2] * (R(1) / R(6));
  const bool trans = C.transverse != 0;
  // the line's values of earlier planes: S, e2p, e2m of plane p-1, e2p of
  // plane p-2, A_z of plane p-1
  R S1[M], e2p1[M], e2m1[M], e2p2[M], Az1[M];
#pragma unroll
  for (int c = 0; c < M; ++c) S1[c] = e2p1[c] = e2m1[c] = e2p2[c] = Az1[c] = R(0);
  R smax = R(0);
  for (int pz = z0 - 1; pz <= z1; ++pz) {
    const int b = NB == 2 ? (pz & 1) : 0;
    R qc[M], ql[M];
    load_cell3<M, R>(C, q, nx, ny, nz, xc, jl, pz, RP::WALL_X, 2, 3, qc);
#pragma unroll
    for (int c = 0; c < M; ++c) {
      ql[c] = __shfl_up_sync(0xffffffffu, qc[c], 1);
      if (lane == 0) ql[c] = qc[c];
    }
    R W[MW][M], s[MW], am[M], ap[M], F[M];
    {
      R x[RP::NCTX];
      RP::template solve<0>(C, ql, qc, nullptr, nullptr, W, s, am, ap, x);
    }
    if (C.order == 2) {
      R dot[MW], nrm[MW];
      constexpr int KS = strength_k<RP, 0>();
#pragma unroll
      for (int p = 0; p < MW; ++p) {
        const bool left = s[p] > R(0);
        if constexpr (KS >= 0) {
          const R wl = __shfl_up_sync(0xffffffffu, W[p][KS], 1);
          const R wr = __shfl_down_sync(0xffffffffu, W[p][KS], 1);
          dot[p] = left ? wl : wr;
          nrm[p] = W[p][KS];
        } else {
          R d_ = R(0), n2 = R(0);
#pragma unroll
          for (int c = 0; c < M; ++c) {
            const R wl = __shfl_up_sync(0xffffffffu, W[p][c], 1);
            const R wr = __shfl_down_sync(0xffffffffu, W[p][c], 1);
            const R up = left ? wl : wr;
            d_ += up * W[p][c];
            n2 += W[p][c] * W[p][c];
          }
          dot[p] = d_;
          nrm[p] = n2;
        }
      }
      correction<RP, R, 0>(C, W, s, dot, nrm, dtdn, F);
    } else {
#pragma unroll
      for (int c = 0; c < M; ++c) F[c] = R(0);
    }
    if (owner_line && interior_line && own_face && pz >= 0 && pz >= z0 && pz < z1) {
#pragma unroll
      for (int p = 0; p < MW; ++p) smax = nanmax(smax, (R)fabs(s[p]));
      const int fx[3] = {f, j, pz};
      const size_t fi = face_index<R>(0, nx, ny, fx);
      st_rec<M, R>(work + L.off_am[0] + fi * M, am);
      st_rec<M, R>(work + L.off_ap[0] + fi * M, ap);
      if (trans) {
        st_rec<M, R>(work + L.off_fc[0] + fi * M, F);
      } else {
        add_fc_own<M, R>(work, L, 0, nx, ny, nz, fx, F);
      }
    }
    if (!trans) continue;
    // cell f: A+dQ - F of face f plus A-dQ + F of face f + 1
    R S[M], e1m[M], e1p[M], e2m[M], e2p[M], Ay[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const R amn = __shfl_down_sync(0xffffffffu, am[c], 1);
      const R Fn = __shfl_down_sync(0xffffffffu, F[c], 1);
      S[c] = (ap[c] - tfF * F[c]) + (amn + tfF * Fn);
    }
    Trans3<RP, R, 1>::split(C, S, e1m, e1p);
    Trans3<RP, R, 2>::split(C, S, e2m, e2p);
#pragma unroll
    for (int c = 0; c < M; ++c) {
      Ay[c] = h * S1[c] + k6z * (e2p1[c] - e2m1[c]) - k6z * (e2p2[c] - e2m[c]);  // plane pz-1
      sh[b][0][c][w][lane] = e1m[c];
      sh[b][1][c][w][lane] = e1p[c];
      sh[b][2][c][w][lane] = Ay[c];
    }
    __syncthreads();
    R Az[M];
    if (w >= 1 && w <= NW - 2) {
#pragma unroll
      for (int c = 0; c < M; ++c)
        Az[c] = h * S[c] + k6y * (e1p[c] - e1m[c]) -
                k6y * (sh[b][1][c][w - 1][lane] - sh[b][0][c][w + 1][lane]);
    } else {
#pragma unroll
      for (int c = 0; c < M; ++c) Az[c] = R(0);
    }
    const int k = pz - 1;
    if (owner_line && own_cell && k >= z0) {
      R Ayu[M], apA[M], amA[M], apB[M], amB[M], v[M];
#pragma unroll
      for (int c = 0; c < M; ++c) Ayu[c] = sh[b][2][c][w + 1][lane];
      // upper y-face of cell (f, j, k)
      Trans3<RP, R, 1>::split(C, Ay, amA, apA);
      Trans3<RP, R, 1>::split(C, Ayu, amB, apB);
#pragma unroll
      for (int c = 0; c < M; ++c) v[c] = apA[c] + amB[c];
      if (k >= 0) {
        const int fy[3] = {f, j + 1, k};
        st_rec<M, R>(work + L.off_fc[1] + face_index<R>(1, nx, ny, fy) * M, v);
      }
      // upper z-face of cell (f, j, k)
      Trans3<RP, R, 2>::split(C, Az1, amA, apA);
      Trans3<RP, R, 2>::split(C, Az, amB, apB);
#pragma unroll
      for (int c = 0; c < M; ++c) v[c] = apA[c] + amB[c];
      if (j >= 0) {
        const int fz[3] = {f, j, k + 1};
        st_rec<M, R>(work + L.off_fc[2] + face_index<R>(2, nx, ny, fz) * M, v);
      }
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
      e2p2[c] = e2p1[c];
      e2p1[c] = e2p[c];
      e2m1[c] = e2m[c];
      S1[c] = S[c];
      Az1[c] = Az[c];
    }
    if (NB == 1) __syncthreads();
  }
  finish_attempt<R>(ctl, smax, R(0), 0, 0, false, R(0));
}

template <class RP, typename R>
__global__ void __launch_bounds__(256)
    classic3d_update(const Member* __restrict__ members, const MConsts<R> C) {
  constexpr int M = RP::M;
  const Member& mb = members[0];
  DevCtl* ctl = mb.ctl;
  __shared__ int s_done, s_cur, s_nbuf;
  __shared__ R s_k[3];
  if (threadIdx.x == 0) {
    s_done = ctl->done;
    s_cur = ctl->cur;
    s_nbuf = ctl->nbuf;
    for (int d = 0; d < 3; ++d) s_k[d] = (R)(ctl->dt / ctl->dx[d]);
  }
  __syncthreads();
  if (s_done) return;
  const int nx = mb.nx, ny = mb.ny, nz = mb.nz;
  const long long ncell = (long long)nx * ny * nz;
  int bad = 0;
  const R* __restrict__ q = (const R*)mb.q[s_cur];
  R* __restrict__ qo = (R*)mb.q[(s_cur + 1) % s_nbuf];
  const R* __restrict__ work = (const R*)mb.work3;
  Faces3 L;
  faces3_layout(nx, ny, nz, M, L);
  // kUpdateCells3d cells per block, consecutive threads on consecutive cells
#pragma unroll
  for (int u = 0; u < kUpdateCells3d / 256; ++u) {
    const long long id = (long long)blockIdx.x * kUpdateCells3d + u * 256 + threadIdx.x;
    if (id >= ncell) break;
    const int i = (int)(id % nx), j = (int)((id / nx) % ny), k = (int)(id / ((long long)nx * ny));
    R v[M];
#pragma unroll
    for (int c = 0; c < M; ++c) v[c] = q[(size_t)c * ncell + id];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      int lo[3] = {i, j, k}, hi[3] = {i, j, k};
      hi[d] += 1;
      const size_t fl = face_index<R>(d, nx, ny, lo), fh = face_index<R>(d, nx, ny, hi);
      const R dtdn = s_k[d];
      R apl[M], amh[M], fch[M], fcl[M];
      ld_rec<M, R>(work + L.off_ap[d] + fl * M, apl);
      ld_rec<M, R>(work + L.off_am[d] + fh * M, amh);
      ld_rec<M, R>(work + L.off_fc[d] + fh * M, fch);
      ld_rec<M, R>(work + L.off_fc[d] + fl * M, fcl);
#pragma unroll
      for (int c = 0; c < M; ++c) v[c] = v[c] - dtdn * (apl[c] + amh[c]) - dtdn * (fch[c] - fcl[c]);
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
      bad |= !isfinite(v[c]);
      qo[(size_t)c * ncell + id] = v[c];
    }
  }
  finish_attempt<R>(ctl, R(0), R(0), bad, mb.ntiles, true, R(0));
}

template <class RP, typename R>
__global__ void __launch_bounds__(256)
    maxspeed3_kernel(const Member* __restrict__ members, const MConsts<R> C) {
  constexpr int M = RP::M, MW = RP::MW;
  const Member& mb = members[0];
  DevCtl* ctl = mb.ctl;
  const int nx = mb.nx, ny = mb.ny, nz = mb.nz;
  const long long ncell = (long long)nx * ny * nz;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  R sm[3] = {R(0), R(0), R(0)};
  if (id < ncell) {
    const int i = (int)(id % nx), j = (int)((id / nx) % ny), k = (int)(id / ((long long)nx * ny));
    const R* q = (const R*)mb.q[ctl->cur];
    const int c3[3] = {i, j, k};
    const int n3[3] = {nx, ny, nz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      for (int side = 0; side < (c3[d] == n3[d] - 1 ? 2 : 1); ++side) {
        int l[3] = {i, j, k}, r[3] = {i, j, k};
        l[d] += side - 1;
        r[d] += side;
        R a[M], b[M], W[MW][M], s[MW], am[M], ap[M], x[RP::NCTX];
        load_cell3<M, R>(C, q, nx, ny, nz, l[0], l[1], l[2], RP::WALL_X, 2, 3, a);
        load_cell3<M, R>(C, q, nx, ny, nz, r[0], r[1], r[2], RP::WALL_X, 2, 3, b);
        if (d == 0) RP::template solve<0>(C, a, b, nullptr, nullptr, W, s, am, ap, x);
        else if (d == 1) RP::template solve<1>(C, a, b, nullptr, nullptr, W, s, am, ap, x);
        else RP::template solve<2>(C, a, b, nullptr, nullptr, W, s, am, ap, x);
#pragma unroll
        for (int p = 0; p < MW; ++p) sm[d] = nanmax(sm[d], (R)fabs(s[p]));
      }
    }
  }
  finish_attempt<R>(ctl, sm[0], sm[1], 0, 0, false, sm[2]);
}

}  // namespace claw
