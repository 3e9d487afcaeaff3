// classic3d.cuh -- 3D unsplit Clawpack-classic step (LeVeque 1997): normal
// solves, limited corrections, transverse and double-transverse propagation,
// for scalar advection and linear acoustics.
//
// One attempt = a zero fill of the per-face arrays, three face sweeps (one per
// direction; a thread walks a segment of faces along the direction with a
// sliding window of waves) that accumulate fluctuations and correction fluxes
// on the faces of interior cells, and an update kernel whose last block runs
// the controller.
// Transverse pieces: a fluctuation a that enters cell c across a d-face adds
// -dt/(2 dx_d) E^+-a to the e-faces of c; the part E^+-a has moved on into
// cell c +- e, so its third-direction split F^+-E^+-a moves 1/6 (dt/dx_d)
// (dt/dx_e) of flux correction from the f-faces of c to those of c +- e
// (six orderings of the directions give the corner-transport-upwind term).
#pragma once

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

template <typename R>
__device__ __forceinline__ size_t face_index(int e, int nx, int ny, const int (&f)[3]) {
  const int NXF = nx + (e == 0), NYF = ny + (e == 1);
  return ((size_t)f[2] * NYF + f[1]) * NXF + f[0];
}

// add coef * v to the correction flux of face f in direction e when it bounds an
// interior cell
template <int M, typename R>
__device__ __forceinline__ void add_fc(R* __restrict__ work, const Faces3& L, int e, int nx,
                                       int ny, int nz, const int (&f)[3], R coef,
                                       const R (&v)[M]) {
  const int n3[3] = {nx, ny, nz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int hi = (d == e) ? n3[d] : n3[d] - 1;
    if (f[d] < 0 || f[d] > hi) return;
  }
  const size_t fi = face_index<R>(e, nx, ny, f);
  R* base = work + L.off_fc[e] + fi * M;
#pragma unroll
  for (int c = 0; c < M; ++c) atomicAdd(base + c, coef * v[c]);
}

// add coef * v to the correction flux of a face this thread alone updates in
// the current launch (a plain read-modify-write; earlier launches' sums are
// already in place by stream order)
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
#pragma unroll
  for (int c = 0; c < M; ++c) base[c] += v[c];
}

// transverse and double-transverse propagation of the fluctuation av that
// enters cell c0 across its faces in direction D (Sec. 2, LeVeque 1997):
// split in each transverse direction e into the four transverse faces of c0
// (summed here, one update per face) and, split again in the third direction
// g, into the g-faces of the cells c0 +- e.  The splits are linear in av, so
// the two fluctuations entering a cell from its two D-faces are propagated
// as one sum.
template <class RP, typename R, int D>
__device__ __forceinline__ void propagate3(const MConsts<R>& C, R* __restrict__ work,
                                           const Faces3& L, int nx, int ny, int nz,
                                           const int (&c0)[3], const R (&av)[RP::M], R dtdn,
                                           const R (&k3)[3]) {
  constexpr int M = RP::M;
  constexpr int E1 = (D + 1) % 3, E2 = (D + 2) % 3;
  R lo1[M], hi1[M], lo2[M], hi2[M];
#pragma unroll
  for (int c = 0; c < M; ++c) lo1[c] = hi1[c] = lo2[c] = hi2[c] = R(0);
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    // transverse direction e and third direction g
    R em[M], ep[M];
    if (t == 0) Trans3<RP, R, E1>::split(C, av, em, ep);
    else Trans3<RP, R, E2>::split(C, av, em, ep);
    const int e = t == 0 ? E1 : E2;
    const int g = t == 0 ? E2 : E1;
    R(&elo)[M] = t == 0 ? lo1 : lo2;
    R(&ehi)[M] = t == 0 ? hi1 : hi2;
    R(&glo)[M] = t == 0 ? lo2 : lo1;
    R(&ghi)[M] = t == 0 ? hi2 : hi1;
    const R h = R(-0.5) * dtdn;
#pragma unroll
    for (int c = 0; c < M; ++c) {
      ehi[c] += h * ep[c];
      elo[c] += h * em[c];
    }
    const R dte = k3[e];
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
      const R(&bv)[M] = sg == 0 ? ep : em;
      const R k6 = (sg == 0 ? R(1) : R(-1)) * dtdn * dte * (R(1) / R(6));
      R gm[M], gp[M];
      if (t == 0) Trans3<RP, R, E2>::split(C, bv, gm, gp);
      else Trans3<RP, R, E1>::split(C, bv, gm, gp);
#pragma unroll
      for (int c = 0; c < M; ++c) {
        ghi[c] += k6 * gp[c];
        glo[c] += k6 * gm[c];
      }
      // the g-faces of the cell the piece moved on to, c0 +- e
      int c2[3] = {c0[0], c0[1], c0[2]};
      c2[e] += sg == 0 ? 1 : -1;
      int fu2[3] = {c2[0], c2[1], c2[2]};
      fu2[g] = c2[g] + 1;
      add_fc<M, R>(work, L, g, nx, ny, nz, fu2, -k6, gp);
      add_fc<M, R>(work, L, g, nx, ny, nz, c2, -k6, gm);
    }
  }
  int u1[3] = {c0[0], c0[1], c0[2]};
  u1[E1] = c0[E1] + 1;
  int u2[3] = {c0[0], c0[1], c0[2]};
  u2[E2] = c0[E2] + 1;
  add_fc<M, R>(work, L, E1, nx, ny, nz, u1, R(1), hi1);
  add_fc<M, R>(work, L, E1, nx, ny, nz, c0, R(1), lo1);
  add_fc<M, R>(work, L, E2, nx, ny, nz, u2, R(1), hi2);
  add_fc<M, R>(work, L, E2, nx, ny, nz, c0, R(1), lo2);
}

// faces along D one sweep thread walks
constexpr int kSweep3dFaces = 16;

template <class RP, typename R, int D>
__global__ void __launch_bounds__(256)
    classic3d_sweep(const Member* __restrict__ members, const MConsts<R> C) {
  constexpr int M = RP::M, MW = RP::MW;
  constexpr int E1 = (D + 1) % 3, E2 = (D + 2) % 3;
  constexpr int T = kSweep3dFaces;
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
  const int nd = n3[D], ne1 = n3[E1], ne2 = n3[E2];
  const int nseg = (nd + 1 + T - 1) / T;
  // segments of T faces along D (faces 0..nd), lines a = -1..ne1, b = -1..ne2
  const long long total = (long long)nseg * (ne1 + 2) * (ne2 + 2);
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  R smax = R(0);
  if (id < total) {
    // x varies fastest across threads (in the x sweep: the segment index)
    int ext[3], v[3];
    ext[D] = nseg;
    ext[E1] = ne1 + 2;
    ext[E2] = ne2 + 2;
    const long long q01 = (long long)ext[0] * ext[1];
    v[0] = (int)(id % ext[0]);
    v[1] = (int)((id / ext[0]) % ext[1]);
    v[2] = (int)(id / q01);
    const int i0 = v[D] * T, i1 = min(i0 + T, nd + 1);
    const int a = v[E1] - 1, b = v[E2] - 1;
    const R* __restrict__ q = (const R*)mb.q[s_cur];
    R* __restrict__ work = (R*)mb.work3;
    Faces3 L;
    faces3_layout(nx, ny, nz, M, L);
    const R dtdn = s_k[D];
    const R k3[3] = {s_k[0], s_k[1], s_k[2]};
    const bool interior_line = a >= 0 && a < ne1 && b >= 0 && b < ne2;
    auto load = [&](int i, R (&out)[M]) {
      int c3[3];
      c3[D] = i;
      c3[E1] = a;
      c3[E2] = b;
      load_cell3<M, R>(C, q, nx, ny, nz, c3[0], c3[1], c3[2], RP::WALL_X, 2, 3, out);
    };
    // window: waves of faces i-1 (Wl), i (Wc) and i+1 (Wr); face i lies
    // between cells i-1 and i
    R Wl[MW][M], Wc[MW][M], Wr[MW][M], sl[MW], sc[MW], sr[MW];
    R amc[M], apc[M], amr[M], apr[M];
    R cl[M], cr[M];
    {
      R x[RP::NCTX], amt[M], apt[M];
      load(i0 - 2, cl);
      load(i0 - 1, cr);
      RP::template solve<D>(C, cl, cr, nullptr, nullptr, Wl, sl, amt, apt, x);
      load(i0, cl);
      RP::template solve<D>(C, cr, cl, nullptr, nullptr, Wc, sc, amc, apc, x);
    }
    // cl holds cell i0 here
    R P[M];  // A+dQ - F of the face left of the current cell (enters it)
    int c0[3];
    c0[E1] = a;
    c0[E2] = b;
    for (int i = i0; i < i1; ++i) {
      {
        R x[RP::NCTX];
        load(i + 1, cr);
        RP::template solve<D>(C, cl, cr, nullptr, nullptr, Wr, sr, amr, apr, x);
#pragma unroll
        for (int c = 0; c < M; ++c) cl[c] = cr[c];
      }
      if (interior_line) {
#pragma unroll
        for (int p = 0; p < MW; ++p) smax = nanmax(smax, (R)fabs(sc[p]));
      }
      R F[M];
      if (C.order == 2) {
        R dot[MW], nrm[MW];
#pragma unroll
        for (int p = 0; p < MW; ++p) {
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
        correction<RP, R, D>(C, Wc, sc, dot, nrm, dtdn, F);
      } else {
#pragma unroll
        for (int c = 0; c < M; ++c) F[c] = R(0);
      }
      if (interior_line) {
        int f[3];
        f[D] = i;
        f[E1] = a;
        f[E2] = b;
        const size_t fi = face_index<R>(D, nx, ny, f);
#pragma unroll
        for (int c = 0; c < M; ++c) {
          work[L.off_am[D] + fi * M + c] = amc[c];
          work[L.off_ap[D] + fi * M + c] = apc[c];
        }
        // within this sweep only this thread touches the D-face's correction
        add_fc_own<M, R>(work, L, D, nx, ny, nz, f, F);
      }
      if (C.transverse) {
        // cell i-1 takes A-dQ + F of face i, plus (inside the segment) the
        // A+dQ - F of face i-1 carried in P
        const R tf = C.transverse == 2 ? R(1) : R(0);
        R av[M];
#pragma unroll
        for (int c = 0; c < M; ++c) av[c] = amc[c] + tf * F[c];
        if (i > i0) {
#pragma unroll
          for (int c = 0; c < M; ++c) av[c] = P[c] + av[c];
        }
        c0[D] = i - 1;
        propagate3<RP, R, D>(C, work, L, nx, ny, nz, c0, av, dtdn, k3);
#pragma unroll
        for (int c = 0; c < M; ++c) P[c] = apc[c] - tf * F[c];
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
    if (C.transverse) {
      // the last face's A+dQ - F enters cell i1-1 (its other face belongs to
      // the next segment)
      c0[D] = i1 - 1;
      propagate3<RP, R, D>(C, work, L, nx, ny, nz, c0, P, dtdn, k3);
    }
  }
  R sx = D == 0 ? smax : R(0), sy = D == 1 ? smax : R(0), sz = D == 2 ? smax : R(0);
  finish_attempt<R>(ctl, sx, sy, 0, 0, false, sz);
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
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int bad = 0;
  if (id < ncell) {
    const int i = (int)(id % nx), j = (int)((id / nx) % ny), k = (int)(id / ((long long)nx * ny));
    const R* __restrict__ q = (const R*)mb.q[s_cur];
    R* __restrict__ qo = (R*)mb.q[(s_cur + 1) % s_nbuf];
    const R* __restrict__ work = (const R*)mb.work3;
    Faces3 L;
    faces3_layout(nx, ny, nz, M, L);
    R v[M];
#pragma unroll
    for (int c = 0; c < M; ++c) v[c] = q[(size_t)c * ncell + id];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      int lo[3] = {i, j, k}, hi[3] = {i, j, k};
      hi[d] += 1;
      const size_t fl = face_index<R>(d, nx, ny, lo), fh = face_index<R>(d, nx, ny, hi);
      const R dtdn = s_k[d];
#pragma unroll
      for (int c = 0; c < M; ++c) {
        v[c] = v[c] - dtdn * (work[L.off_ap[d] + fl * M + c] + work[L.off_am[d] + fh * M + c]) -
               dtdn * (work[L.off_fc[d] + fh * M + c] - work[L.off_fc[d] + fl * M + c]);
      }
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
