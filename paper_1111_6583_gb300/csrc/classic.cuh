// classic.cuh -- fused Clawpack-classic step kernels.
//
// One launch = one attempt of one step for every member of a tile table:
// ghost-cell remap in the loads, Riemann solve at every interface, wave
// limiting, second-order corrections (Eq. (lwflux)), transverse corrections in
// 2D (Sec. 3.1; LeVeque 1997), conservative update (Eq. (fluxdiff)) and the
// per-block maximum wave speed; the last block of a member runs the CFL
// controller (Sec. 5).
#pragma once

#include "riemann.cuh"

namespace claw {


// ---------------------------------------------------------------------------
// 1D: a block loads T + 4 cells (2 ghosts each side) into shared memory,
// solves T + 3 Riemann problems, limits T + 1 interfaces and updates T cells.
// ---------------------------------------------------------------------------
template <class RP, typename R, int NT, int T>
__global__ void __launch_bounds__(NT)
    classic1d_kernel(const Member* __restrict__ members, const Tile* __restrict__ tiles,
                     int ntiles_total, const MConsts<R> C) {
  constexpr int M = RP::M, MW = RP::MW, MA = RP::MA;
  constexpr int MAS = MA > 0 ? MA : 1;
  __shared__ R qs[M][T + 4];
  __shared__ R as[MAS][MA > 0 ? T + 4 : 1];
  __shared__ R Ws[MW][M][T + 3];
  __shared__ R Ss[MW][T + 3];
  __shared__ R Am[M][T + 1];
  __shared__ R Ap[M][T + 1];
  __shared__ int s_done, s_cur, s_nbuf;
  __shared__ double s_dt;

  for (int it = blockIdx.x; it < ntiles_total; it += gridDim.x) {
    const Tile tl = tiles ? tiles[it] : Tile{0, it};
    const Member& mb = members[tl.member];
    DevCtl* ctl = mb.ctl;
    if (threadIdx.x == 0) {
      s_done = ctl->done;
      s_dt = ctl->dt;
      s_cur = ctl->cur;
      s_nbuf = ctl->nbuf;
    }
    __syncthreads();
    if (s_done) {
      __syncthreads();
      continue;
    }
    const int nx = mb.nx;
    const int i0 = tl.tile * T;
    const int cnt = min(T, nx - i0);
    const R* __restrict__ q = (const R*)mb.q[s_cur];
    R* __restrict__ qo = (R*)mb.q[(s_cur + 1) % s_nbuf];
    const R* __restrict__ aux = (const R*)mb.aux;
    const R dtdx = (R)(s_dt / ctl->dx[0]);

    // stage cells i0-2 .. i0+cnt+1 (ghosts by index remap)
    for (int j = threadIdx.x; j < cnt + 4; j += NT) {
      R v[M];
      load_cell<M, R>(C, q, nx, 1, i0 - 2 + j, 0, RP::WALL_X, -1, v);
#pragma unroll
      for (int k = 0; k < M; ++k) qs[k][j] = v[k];
      if (MA > 0) {
        R a[MAS];
        load_aux<MA, R>(C, aux, nx, 1, i0 - 2 + j, 0, a);
#pragma unroll
        for (int k = 0; k < MA; ++k) as[k][j] = a[k];
      }
    }
    __syncthreads();

    // Riemann problems at interfaces i0-1 .. i0+cnt+1 (index ii = i - i0 + 1)
    double smax = 0.0;
    for (int ii = threadIdx.x; ii < cnt + 3; ii += NT) {
      R ql[M], qr[M], al[MAS], ar[MAS];
#pragma unroll
      for (int k = 0; k < M; ++k) {
        ql[k] = qs[k][ii];
        qr[k] = qs[k][ii + 1];
      }
#pragma unroll
      for (int k = 0; k < MA; ++k) {
        al[k] = as[k][ii];
        ar[k] = as[k][ii + 1];
      }
      R W[MW][M], s[MW], am[M], ap[M], ctx[RP::NCTX];
      RP::template solve<0>(C, ql, qr, al, ar, W, s, am, ap, ctx);
#pragma unroll
      for (int p = 0; p < MW; ++p) {
        Ss[p][ii] = s[p];
#pragma unroll
        for (int k = 0; k < M; ++k) Ws[p][k][ii] = W[p][k];
      }
      if (ii >= 1 && ii <= cnt + 1) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          Am[k][ii - 1] = am[k];
          Ap[k][ii - 1] = ap[k];
        }
#pragma unroll
        for (int p = 0; p < MW; ++p) smax = nanmax(smax, (double)fabs(s[p]));
      }
    }
    __syncthreads();

    // limited corrections at interfaces i0 .. i0+cnt, folded into the
    // fluctuations: cell i gets -dt/dx (A^+dQ_i - F_i) and -dt/dx (A^-dQ_{i+1} + F_{i+1})
    if (C.order == 2) {
      for (int jj = threadIdx.x; jj < cnt + 1; jj += NT) {
        const int ii = jj + 1;
        R W[MW][M], s[MW], dot[MW], nrm[MW], F[M];
#pragma unroll
        for (int p = 0; p < MW; ++p) {
          s[p] = Ss[p][ii];
          const int iu = s[p] > R(0) ? ii - 1 : ii + 1;
          R d = R(0), n2 = R(0);
#pragma unroll
          for (int k = 0; k < M; ++k) {
            W[p][k] = Ws[p][k][ii];
            d += Ws[p][k][iu] * W[p][k];
            n2 += W[p][k] * W[p][k];
          }
          dot[p] = d;
          nrm[p] = n2;
        }
        correction<RP, R>(C, W, s, dot, nrm, dtdx, F);
#pragma unroll
        for (int k = 0; k < M; ++k) {
          Ap[k][jj] -= F[k];
          Am[k][jj] += F[k];
        }
      }
      __syncthreads();
    }

    // conservative update of cells i0 .. i0+cnt-1
    int bad = 0;
    const size_t plane = (size_t)nx;
    for (int j = threadIdx.x; j < cnt; j += NT) {
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const R v = qs[k][j + 2] - dtdx * (Ap[k][j] + Am[k][j + 1]);
        bad |= !isfinite(v);
        qo[k * plane + i0 + j] = v;
      }
    }
    finish_attempt(ctl, smax, 0.0, bad, mb.ntiles, true);
  }
}

// ---------------------------------------------------------------------------
// 2D unsplit step.  A block of BW threads owns a strip of BW-4 interior
// columns and walks down H interior rows of it.  Thread l holds column
// c = c0 - 2 + l.  Per row R it solves the x-interface (c, R) and the
// y-interface between rows R-1 and R, limits the x-interface with its lane
// neighbours' waves and the y-interface R-1 with the waves of the rows above
// and below (kept in registers), applies transverse corrections, and
// scatters every contribution into per-cell accumulators of rows R-2 .. R+1
// (own column in registers, neighbour columns through shared-memory
// mailboxes).  Row R-2 is then complete and is written out.
// ---------------------------------------------------------------------------
template <class RP, typename R, int BW>
__global__ void __launch_bounds__(BW)
    classic2d_kernel(const Member* __restrict__ members, const Tile* __restrict__ tiles,
                     int ntiles_total, const MConsts<R> C, int H) {
  constexpr int M = RP::M, MW = RP::MW, NC = RP::NCTX;
  constexpr int TX = BW - 4;
  __shared__ R qs[M][BW];
  __shared__ R xws[MW][M][BW];
  __shared__ R mbl[4][M][BW];
  __shared__ R mbr[2][M][BW];
  __shared__ int s_done, s_cur, s_nbuf;
  __shared__ double s_dt;
  const int l = threadIdx.x;

  for (int it = blockIdx.x; it < ntiles_total; it += gridDim.x) {
    const Tile tl = tiles ? tiles[it] : Tile{0, it};
    const Member& mb = members[tl.member];
    DevCtl* ctl = mb.ctl;
    if (l == 0) {
      s_done = ctl->done;
      s_dt = ctl->dt;
      s_cur = ctl->cur;
      s_nbuf = ctl->nbuf;
    }
    __syncthreads();
    if (s_done) {
      __syncthreads();
      continue;
    }
    const int nx = mb.nx, ny = mb.ny;
    const int nsx = (nx + TX - 1) / TX;
    const int c0 = (tl.tile % nsx) * TX;
    const int r0 = (tl.tile / nsx) * H;
    const int rend = min(r0 + H, ny) - 1;
    const int c = c0 - 2 + l;
    const int cload = min(c, nx + 1);
    const bool col_in = (l >= 2) && (l < BW - 2) && (c < nx);
    const bool xlim = (l >= 2) && (l <= BW - 2);
    const bool xcfl = xlim && (c <= nx);
    const bool ylim = (l >= 1) && (l <= BW - 2);
    const R* __restrict__ q = (const R*)mb.q[s_cur];
    R* __restrict__ qo = (R*)mb.q[(s_cur + 1) % s_nbuf];
    const double dtd = s_dt;
    const R dtdx = (R)(dtd / ctl->dx[0]);
    const R dtdy = (R)(dtd / ctl->dx[1]);
    const R kxy = (R)(0.5 * (dtd / ctl->dx[0]) * (dtd / ctl->dx[1]));
    const size_t plane = (size_t)nx * ny;

    R qm2[M], qm1[M], qc[M];
    R acc0[M], acc1[M], acc2[M], acc3[M];
    // y-interface R-1 (previous): waves, speeds, fluctuations, linearisation,
    // norms and dot products with the interface below it
    R yW[MW][M], ys[MW], yam[M], yap[M], yx[NC], ynrm[MW], ydot[MW];
#pragma unroll
    for (int k = 0; k < M; ++k) {
      qc[k] = qm1[k] = R(0);
      acc0[k] = acc1[k] = acc2[k] = acc3[k] = R(0);
      yam[k] = yap[k] = R(0);
    }
#pragma unroll
    for (int p = 0; p < MW; ++p) {
      ys[p] = ynrm[p] = ydot[p] = R(0);
#pragma unroll
      for (int k = 0; k < M; ++k) yW[p][k] = R(0);
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) yx[k] = R(0);
    double smx = 0.0, smy = 0.0;
    int bad = 0;

    for (int Rw = r0 - 2; Rw <= rend + 2; ++Rw) {
      // (1) load row Rw
#pragma unroll
      for (int k = 0; k < M; ++k) {
        qm2[k] = qm1[k];
        qm1[k] = qc[k];
      }
      load_cell<M, R>(C, q, nx, ny, cload, Rw, RP::WALL_X, RP::WALL_Y, qc);
#pragma unroll
      for (int k = 0; k < M; ++k) qs[k][l] = qc[k];

      // (2) y-interface Rw (rows Rw-1, Rw)
      R nW[MW][M], ns[MW], nam[M], nap[M], nx_[NC], nnrm[MW], ndot[MW];
      const bool yrow = Rw >= r0 - 1;
      if (yrow) {
        RP::template solve<1>(C, qm1, qc, nullptr, nullptr, nW, ns, nam, nap, nx_);
#pragma unroll
        for (int p = 0; p < MW; ++p) {
          R a = R(0), b = R(0);
#pragma unroll
          for (int k = 0; k < M; ++k) {
            a += nW[p][k] * nW[p][k];
            b += nW[p][k] * yW[p][k];
          }
          nnrm[p] = a;
          ndot[p] = b;
        }
        if (col_in && Rw >= r0 && Rw <= rend + 1) {
#pragma unroll
          for (int p = 0; p < MW; ++p) smy = nanmax(smy, (double)fabs(ns[p]));
        }
      }
      __syncthreads();  // qs ready

      // (3) x-interface (c, Rw)
      const bool xrow = (Rw >= r0 - 1) && (Rw <= rend + 1);
      R xW[MW][M], xs[MW], xam[M], xap[M], xx[NC];
      if (xrow && l >= 1) {
        R ql[M];
#pragma unroll
        for (int k = 0; k < M; ++k) ql[k] = qs[k][l - 1];
        RP::template solve<0>(C, ql, qc, nullptr, nullptr, xW, xs, xam, xap, xx);
#pragma unroll
        for (int p = 0; p < MW; ++p)
#pragma unroll
          for (int k = 0; k < M; ++k) xws[p][k][l] = xW[p][k];
      }
      __syncthreads();  // x waves ready

      R tl_[4][M], tr_[2][M];
#pragma unroll
      for (int k = 0; k < M; ++k) {
        tl_[0][k] = tl_[1][k] = tl_[2][k] = tl_[3][k] = R(0);
        tr_[0][k] = tr_[1][k] = R(0);
      }

      // (4) x-limiting, corrections, transverse propagation
      if (xrow && xlim) {
        R F[M];
        if (C.order == 2) {
          R dot[MW], nrm[MW];
#pragma unroll
          for (int p = 0; p < MW; ++p) {
            const int lu = xs[p] > R(0) ? l - 1 : l + 1;
            R a = R(0), b = R(0);
#pragma unroll
            for (int k = 0; k < M; ++k) {
              b += xws[p][k][lu] * xW[p][k];
              a += xW[p][k] * xW[p][k];
            }
            dot[p] = b;
            nrm[p] = a;
          }
          correction<RP, R>(C, xW, xs, dot, nrm, dtdx, F);
        } else {
#pragma unroll
          for (int k = 0; k < M; ++k) F[k] = R(0);
        }
        R ap_[M], am_[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
          ap_[k] = xap[k] - F[k];
          am_[k] = xam[k] + F[k];
          acc2[k] -= dtdx * ap_[k];
          tl_[2][k] -= dtdx * am_[k];
        }
        if (xcfl && Rw >= r0 && Rw <= rend) {
#pragma unroll
          for (int p = 0; p < MW; ++p) smx = nanmax(smx, (double)fabs(xs[p]));
        }
        if (C.transverse) {
          R tp[M], tm[M], bmp[M], bpp[M], bmm[M], bpm[M];
#pragma unroll
          for (int k = 0; k < M; ++k) {
            tp[k] = C.transverse == 2 ? ap_[k] : xap[k];
            tm[k] = C.transverse == 2 ? am_[k] : xam[k];
          }
          RP::template trans<0>(C, xx, tp, bmp, bpp);
          RP::template trans<0>(C, xx, tm, bmm, bpm);
#pragma unroll
          for (int k = 0; k < M; ++k) {
            acc2[k] += kxy * (bpp[k] - bmp[k]);
            acc3[k] -= kxy * bpp[k];
            acc1[k] += kxy * bmp[k];
            tl_[2][k] += kxy * (bpm[k] - bmm[k]);
            tl_[3][k] -= kxy * bpm[k];
            tl_[1][k] += kxy * bmm[k];
          }
        }
      }

      // (5) y-limiting of interface Rw-1, corrections, transverse propagation
      if (ylim && Rw - 1 >= r0 && Rw - 1 <= rend + 1) {
        R G[M];
        if (C.order == 2) {
          R dot[MW];
#pragma unroll
          for (int p = 0; p < MW; ++p) dot[p] = ys[p] > R(0) ? ydot[p] : ndot[p];
          correction<RP, R>(C, yW, ys, dot, ynrm, dtdy, G);
        } else {
#pragma unroll
          for (int k = 0; k < M; ++k) G[k] = R(0);
        }
        R bp_[M], bm_[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
          bp_[k] = yap[k] - G[k];
          bm_[k] = yam[k] + G[k];
          acc1[k] -= dtdy * bp_[k];
          acc0[k] -= dtdy * bm_[k];
        }
        if (C.transverse) {
          R tp[M], tm[M], amp[M], app[M], amm[M], apm[M];
#pragma unroll
          for (int k = 0; k < M; ++k) {
            tp[k] = C.transverse == 2 ? bp_[k] : yap[k];
            tm[k] = C.transverse == 2 ? bm_[k] : yam[k];
          }
          RP::template trans<1>(C, yx, tp, amp, app);
          RP::template trans<1>(C, yx, tm, amm, apm);
#pragma unroll
          for (int k = 0; k < M; ++k) {
            acc1[k] += kxy * (app[k] - amp[k]);
            acc0[k] += kxy * (apm[k] - amm[k]);
            tr_[1][k] -= kxy * app[k];
            tr_[0][k] -= kxy * apm[k];
            tl_[1][k] += kxy * amp[k];
            tl_[0][k] += kxy * amm[k];
          }
        }
      }
#pragma unroll
      for (int k = 0; k < M; ++k) {
        mbl[0][k][l] = tl_[0][k];
        mbl[1][k][l] = tl_[1][k];
        mbl[2][k][l] = tl_[2][k];
        mbl[3][k][l] = tl_[3][k];
        mbr[0][k][l] = tr_[0][k];
        mbr[1][k][l] = tr_[1][k];
      }
      __syncthreads();  // mailboxes ready

      // (6) gather neighbour contributions, (7) finish row Rw-2
      if (l + 1 < BW) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          acc0[k] += mbl[0][k][l + 1];
          acc1[k] += mbl[1][k][l + 1];
          acc2[k] += mbl[2][k][l + 1];
          acc3[k] += mbl[3][k][l + 1];
        }
      }
      if (l >= 1) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          acc0[k] += mbr[0][k][l - 1];
          acc1[k] += mbr[1][k][l - 1];
        }
      }
      const int Rf = Rw - 2;
      if (col_in && Rf >= r0 && Rf <= rend) {
        const size_t off = (size_t)Rf * nx + c;
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const R v = qm2[k] + acc0[k];
          bad |= !isfinite(v);
          qo[k * plane + off] = v;
        }
      }
#pragma unroll
      for (int k = 0; k < M; ++k) {
        acc0[k] = acc1[k];
        acc1[k] = acc2[k];
        acc2[k] = acc3[k];
        acc3[k] = R(0);
      }
      if (yrow) {
#pragma unroll
        for (int p = 0; p < MW; ++p) {
          ys[p] = ns[p];
          ynrm[p] = nnrm[p];
          ydot[p] = ndot[p];
#pragma unroll
          for (int k = 0; k < M; ++k) yW[p][k] = nW[p][k];
        }
#pragma unroll
        for (int k = 0; k < M; ++k) {
          yam[k] = nam[k];
          yap[k] = nap[k];
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) yx[k] = nx_[k];
      }
    }
    finish_attempt(ctl, smx, smy, bad, mb.ntiles, true);
  }
}

}  // namespace claw
