// sharpclaw.cuh -- fused SharpClaw stage kernel (Sec. 2 method of lines;
// Sec. 2.1: WENO reconstruction, normal Riemann problems only in multi-D).
//
// One launch = one Runge-Kutta stage for every member of a tile table.  A
// block stages a TX x TY tile of Q^(k) plus an RW-cell halo (ghost remap in
// the load), reconstructs left/right interface values by WENO of order
// 2 RW - 1 (component- or
// characteristic-wise, projection at the Roe state of each interface), solves
// the interface Riemann problems and the in-cell problems (total fluctuation
// A dQ_i), forms L(Q) = -(A^+dQ_{i-1/2} + A^-dQ_{i+1/2} + A dQ_i)/dx summed
// over directions, and writes the stage's linear combinations (StageOp: the
// Shu-Osher SSP-RK3 or the low-storage SSP(10,4) stages).  The last stage's
// last block runs the CFL controller.
#pragma once

#include <type_traits>

#include "async_copy.cuh"
#include "kernels.h"
#include "riemann.cuh"
#include "weno_hi.cuh"

namespace claw {

// Both Jiang-Shu WENO5 values at the interface between cells c and d of the
// six cell averages a..f: the left-biased one at the right edge of c (um)
// and the right-biased one at the left edge of d (up), as numerator and
// denominator.  The two use the same candidates from stencils (b, c, d) and
// (c, d, e) and the same second differences of those stencils, computed
// once here; candidates are kept times 6 (the 6 moves to the denominator).
template <typename R>
__device__ __forceinline__ void weno5_pair(R a, R b, R c, R d, R e, R f, R eps, R& nm, R& dm,
                                           R& np, R& dp) {
  const R p0 = R(2) * a - R(7) * b + R(11) * c;   // (a, b, c) at the right edge of c
  const R p1 = R(2) * d + R(5) * c - b;           // (b, c, d) at the c|d edge
  const R p2 = R(2) * c + R(5) * d - e;           // (c, d, e) at the c|d edge
  const R p3 = R(2) * f - R(7) * e + R(11) * d;   // (d, e, f) at the left edge of d
  const R k13 = R(13) / R(12);
  const R t0 = a - R(2) * b + c, t1 = b - R(2) * c + d, t2 = c - R(2) * d + e,
          t3 = d - R(2) * e + f;
  const R h0 = k13 * (t0 * t0), h1 = k13 * (t1 * t1), h2 = k13 * (t2 * t2),
          h3 = k13 * (t3 * t3);
  const R u0 = a - R(4) * b + R(3) * c, u1 = b - d, u2 = R(3) * c - R(4) * d + e;
  const R v0 = f - R(4) * e + R(3) * d, v1 = e - c, v2 = R(3) * d - R(4) * c + b;
  const R e0 = eps + (h0 + R(0.25) * (u0 * u0)), e1 = eps + (h1 + R(0.25) * (u1 * u1)),
          e2 = eps + (h2 + R(0.25) * (u2 * u2));
  const R g0 = eps + (h3 + R(0.25) * (v0 * v0)), g1 = eps + (h2 + R(0.25) * (v1 * v1)),
          g2 = eps + (h1 + R(0.25) * (v2 * v2));
  // alpha_k = d_k / beta_k^2 multiplied through by the product of the three
  const R s0 = e0 * e0, s1 = e1 * e1, s2 = e2 * e2;
  const R w0 = R(0.1) * (s1 * s2), w1 = R(0.6) * (s0 * s2), w2 = R(0.3) * (s0 * s1);
  nm = w0 * p0 + w1 * p1 + w2 * p2;
  dm = R(6) * (w0 + w1 + w2);
  const R z0 = g0 * g0, z1 = g1 * g1, z2 = g2 * g2;
  const R y0 = R(0.1) * (z1 * z2), y1 = R(0.6) * (z0 * z2), y2 = R(0.3) * (z0 * z1);
  np = y0 * p3 + y1 * p2 + y2 * p1;
  dp = R(6) * (y0 + y1 + y2);
}

// n / d for N pairs.  In FP64 with one division: 1/d_i = (prod_{j<i} d_j)
// (prod_{j>i} d_j) / prod_j d_j, taken only when every partial product is a
// positive normal number (no overflow, underflow or lost precision), else N
// divisions.
template <typename R, int N>
__device__ __forceinline__ void div_many(const R (&n)[N], const R (&d)[N], R (&q)[N]) {
  if constexpr (sizeof(R) == 8 && N > 1) {
    R pre[N];
    R prod = d[0];
    bool normal = pos_normal(prod);
    pre[0] = R(1);
#pragma unroll
    for (int i = 1; i < N; ++i) {
      pre[i] = prod;
      prod = prod * d[i];
      normal = normal && pos_normal(prod);
    }
    if (normal) {
      R suf = FM<R>::rcp(prod);
#pragma unroll
      for (int i = N - 1; i >= 0; --i) {
        q[i] = n[i] * (i == 0 ? suf : suf * pre[i]);
        suf = suf * d[i];
      }
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) q[i] = FM<R>::div(n[i], d[i]);
}

// WENO of order 2 RW - 1 (7 .. 17; WENO5 takes weno5_pair): left-biased value at the right edge of cell
// v[o + RW - 1] from v[o .. o + 2 RW - 2] (REV: the mirrored stencil, value at
// the left edge of cell v[o + RW], read from v[o + 2 RW - 1] downwards).
template <int RW, bool REV, typename R, int NV>
__device__ __forceinline__ R weno_edge(const R (&w)[NV], R eps) {
  constexpr int n = 2 * RW - 1;
  R v[n];
#pragma unroll
  for (int j = 0; j < n; ++j) v[j] = REV ? w[n - j] : w[j];
  if constexpr (RW == 4) return weno7<R>(v, eps);
  else if constexpr (RW == 5) return weno9<R>(v, eps);
  else if constexpr (RW == 6) return weno11<R>(v, eps);
  else if constexpr (RW == 7) return weno13<R>(v, eps);
  else if constexpr (RW == 8) return weno15<R>(v, eps);
  else return weno17<R>(v, eps);
}

// static shared memory of sharp_stage_kernel (the arrays declared in it)
template <class RP, typename R, int ND, int TX, int TY, int RW>
constexpr size_t sharp_smem_bytes() {
  constexpr int M = RP::M, MA = RP::MA, G = RW;
  constexpr int MAS = MA > 0 ? MA : 1;
  constexpr int HX = TX + 2 * G, HY = (ND == 2) ? TY + 2 * G : 1;
  constexpr bool kStageRows = TX * TY <= 128;
  constexpr int A = 16 / (int)sizeof(R), OX = kStageRows ? (A - G % A) % A : 0;
  constexpr int HXP0 = (OX + HX + A - 1) / A * A;
  constexpr int HXP = !kStageRows ? HX : ((HXP0 / A) % 2 == 1 ? HXP0 : HXP0 + A);
  constexpr int NE = (ND == 2) ? (TX + 1) * TY + TX * (TY + 1) : TX + 1;
  return sizeof(R) * ((size_t)M * HY * HXP + (size_t)MAS * (MA > 0 ? HY * HXP : 1) +
                      (size_t)HY * HX + 4 * (size_t)M * NE + 3) +
         3 * sizeof(int) + 8;
}

template <class RP, typename R, int ND, int TX, int TY, int RW>
__global__ void __launch_bounds__(TX * TY)
    sharp_stage_kernel(const Member* __restrict__ members, const Tile* __restrict__ tiles,
                       int ntiles_total, const MConsts<R> C, const StageOp op) {
  constexpr int M = RP::M, MW = RP::MW, MA = RP::MA, NC = RP::NCTX;
  constexpr int MAS = MA > 0 ? MA : 1;
  constexpr int NT = TX * TY;
  constexpr int G = RW;        // ghost / halo width
  constexpr int NS = 2 * RW;   // cells around an interface
  constexpr int HX = TX + 2 * G, HY = (ND == 2) ? TY + 2 * G : 1;
  // interface slots: the x-interfaces (TX + 1 per row) first, then the
  // y-interfaces (TY + 1 per column)
  constexpr int NEX = (ND == 2) ? (TX + 1) * TY : TX + 1;
  constexpr int NEY = (ND == 2) ? TX * (TY + 1) : 0;
  constexpr int NE = NEX + NEY;
  // staged rows: a tile row of a field is HXP values from the 16-byte
  // boundary at or below the halo's first cell; cell hi of the halo sits at
  // column OX + hi (tiles start at multiples of TX, a multiple of A)
  // Staged rows, for tiles of 128 threads or fewer (with 256-thread tiles
  // the staging state spilled and the copies measured slower than the
  // cell-by-cell loads in FP32: 0.64-0.71 against 0.61 ms per shock-bubble
  // step); rows padded to an odd number of 16-byte units, so that a column
  // of cells spreads over the shared-memory banks (the y-interface phase
  // reads down columns).  Without staging the rows are HX values, OX = 0.
  constexpr bool kStageRows = NT <= 128;
  constexpr int A = 16 / (int)sizeof(R), OX = kStageRows ? (A - G % A) % A : 0;
  constexpr int HXP0 = (OX + HX + A - 1) / A * A;
  constexpr int HXP = !kStageRows ? HX : ((HXP0 / A) % 2 == 1 ? HXP0 : HXP0 + A);
  static_assert(!kStageRows || TX % A == 0, "tile columns start on 16-byte boundaries");
  __shared__ __align__(16) R Qt[M][HY][HXP];
  __shared__ __align__(16) R At[MAS][MA > 0 ? HY : 1][MA > 0 ? HXP : 1];
  __shared__ __align__(8) unsigned long long s_bar;  // completes the staging copies
  __shared__ R Kt[HY][HX];  // capacity kappa (when the method has one)
  __shared__ R EL[M][NE];  // left edge value of the cell right of an interface
  __shared__ R ER[M][NE];  // right edge value of the cell left of an interface
  __shared__ R FM[M][NE];  // A^- dQ at the interface
  __shared__ R FP[M][NE];  // A^+ dQ at the interface
  __shared__ int s_done, s_cur, s_nbuf;
  __shared__ R s_dt, s_idn[2];

  const int tid = threadIdx.x;
  const int ti = tid % TX, tj = tid / TX;
  [[maybe_unused]] unsigned phase = 0u;  // parity of the staging barrier's phase
  if constexpr (kStageRows) {
    if (tid == 0) {
      mbar_init(smem_u32(&s_bar), 1u);
      fence_mbar_init();
    }
  }

  for (int it = blockIdx.x; it < ntiles_total; it += gridDim.x) {
    const Tile tl = tiles ? tiles[it] : Tile{0, it};
    const Member& mb = members[tl.member];
    DevCtl* ctl = mb.ctl;
    if (tid == 0) {
      s_done = ctl->done;
      s_dt = (R)ctl->dt;
      s_idn[0] = (R)(1.0 / ctl->dx[0]);
      s_idn[1] = (R)(1.0 / ctl->dx[1]);
      s_cur = ctl->cur;
      s_nbuf = ctl->nbuf;
    }
    __syncthreads();
    if (s_done) {
      __syncthreads();
      continue;
    }
    const int nx = mb.nx, ny = (ND == 2) ? mb.ny : 1;
    const int nsx = (nx + TX - 1) / TX;
    const int c0 = (tl.tile % nsx) * TX;
    const int r0 = (ND == 2) ? (tl.tile / nsx) * TY : 0;
    const int cur = s_cur;
    const int nb = s_nbuf;
    const R* __restrict__ qk = (const R*)step_input(mb, cur, nb, op.in);
    const R* __restrict__ qa = (const R*)step_input(mb, cur, nb, op.sa);
    const R* __restrict__ qb = (const R*)step_input(mb, cur, nb, op.sb);
    R* __restrict__ qo = (R*)mb.q[(cur + op.out) % nb];
    R* __restrict__ qo2 = op.out2 >= 0 ? (R*)mb.q[(cur + op.out2) % nb] : nullptr;
    const R* __restrict__ aux = (const R*)mb.aux;
    const size_t plane = (size_t)nx * ny;

    // stage Q^(k) (and aux) with a G-cell halo.  A tile whose halo rows lie
    // inside the grid, with 16-byte aligned fields and rows, arrives by
    // bulk asynchronous copies, one per row and field (HXP values each, the
    // corners and the padding included), completing on the block's
    // barrier; the others (and methods with a capacity field) are loaded
    // cell by cell with the ghost-cell remap, corners skipped in 2D.
    int bad = 0;
    const int xa = c0 - G - OX;  // first staged column
    bool staged = false;
    if constexpr (kStageRows)
      staged = C.capa < 0 && xa >= 0 && xa + HXP <= nx &&
               (ND == 1 || (r0 - G >= 0 && r0 + TY + G <= ny)) &&
               ((size_t)nx * sizeof(R)) % 16 == 0 && ((size_t)qk & 15) == 0 &&
               (MA == 0 || ((size_t)aux & 15) == 0);
    if (staged) {
      const unsigned bar = smem_u32(&s_bar);
      constexpr int NCP = (M + MA) * HY;
      constexpr unsigned RB = HXP * sizeof(R);
      if (tid == 0) mbar_arrive_expect_tx(bar, NCP * RB);
      // a block's later tile refills rows that its previous tile read
      // (those reads precede the barriers of finish_attempt)
      if (it != (int)blockIdx.x && tid < NCP) fence_proxy_async_smem();
      for (int cp = tid; cp < NCP; cp += NT) {
        const int f = cp / HY, hj = cp % HY;
        const int r = (ND == 2) ? r0 - G + hj : 0;
        const R* src = f < M ? qk + (size_t)f * plane + (size_t)r * nx + xa
                             : aux + (size_t)(f - M) * plane + (size_t)r * nx + xa;
        R* dst = f < M ? &Qt[f][hj][0] : &At[MA > 0 ? f - M : 0][MA > 0 ? hj : 0][0];
        bulk_g2s(smem_u32(dst), src, RB, bar);
      }
      const bool got = mbar_wait_bounded(bar, phase);
      if (__syncthreads_or(!got)) {
        // a copy did not complete in time: wait (bounded) for the rest,
        // report CLAW_ETIMEOUT through the control block, compute nothing
        mbar_wait_bounded(bar, phase);
        bad = 2;
      }
      phase ^= 1u;
    } else {
      for (int idx = tid; idx < HX * HY; idx += NT) {
        const int hi = idx % HX, hj = idx / HX;
        if (ND == 2) {
          const bool xin = hi >= G && hi < G + TX, yin = hj >= G && hj < G + TY;
          if (!xin && !yin) continue;
        }
        const int c = c0 - G + hi, r = (ND == 2) ? r0 - G + hj : 0;
        R v[M];
        load_cell<M, R>(C, qk, nx, ny, min(c, nx + G - 1), (ND == 2) ? min(r, ny + G - 1) : 0,
                        RP::WALL_X, RP::WALL_Y, v);
#pragma unroll
        for (int k = 0; k < M; ++k) Qt[k][hj][OX + hi] = v[k];
        if (MA > 0) {
          R a[MAS];
          load_aux<MA, R>(C, aux, nx, ny, min(c, nx + G - 1),
                          (ND == 2) ? min(r, ny + G - 1) : 0, a);
#pragma unroll
          for (int k = 0; k < MA; ++k) At[k][MA > 0 ? hj : 0][MA > 0 ? OX + hi : 0] = a[k];
        }
        if (C.capa >= 0)
          Kt[hj][hi] = load_aux_field<R>(C, aux, nx, ny, min(c, nx + G - 1),
                                         (ND == 2) ? min(r, ny + G - 1) : 0, C.capa);
      }
      __syncthreads();
    }
    const bool skip = bad != 0;

    R L[M];
#pragma unroll
    for (int k = 0; k < M; ++k) L[k] = R(0);
    R smx = R(0), smy = R(0);

    // (a, b) every interface of both directions, each by one thread:
    // reconstruction of its two edge values, then its Riemann problem
    // (q^R_{a-1}, q^L_a) from the same thread's edge values
    auto interface = [&](auto dirc, int le, int e) {
      constexpr int dir = decltype(dirc)::value;
      const int na = (dir == 0) ? TX + 1 : TY + 1;
      const int a = le % na, b = le / na;
      R cell[NS][M];
#pragma unroll
      for (int k6 = 0; k6 < NS; ++k6) {
        // cells a-RW .. a+RW-1 along the line
        const int hi = (dir == 0) ? a + k6 : G + b;
        const int hj = (dir == 0) ? ((ND == 2) ? G + b : 0) : a + k6;
#pragma unroll
        for (int k = 0; k < M; ++k) cell[k6][k] = Qt[k][hj][OX + hi];
      }
      R wm[M], wp[M];
      if (C.char_decomp) {
        R x[NC];
        R w[NS][M];
        RP::template char_ctx<dir>(C, cell[RW - 1], cell[RW], x);
#pragma unroll
        for (int k6 = 0; k6 < NS; ++k6) RP::template to_char<dir>(C, x, cell[k6], w[k6]);
        R um[M], up[M];
        if constexpr (RW == 3) {
          R nn[2 * M], dd[2 * M], vv[2 * M];
#pragma unroll
          for (int k = 0; k < M; ++k)
            weno5_pair<R>(w[0][k], w[1][k], w[2][k], w[3][k], w[4][k], w[5][k], C.weno_eps,
                          nn[k], dd[k], nn[M + k], dd[M + k]);
          div_many<R, 2 * M>(nn, dd, vv);
#pragma unroll
          for (int k = 0; k < M; ++k) {
            um[k] = vv[k];
            up[k] = vv[M + k];
          }
        } else {
#pragma unroll
          for (int k = 0; k < M; ++k) {
            R line[NS];
#pragma unroll
            for (int k6 = 0; k6 < NS; ++k6) line[k6] = w[k6][k];
            um[k] = weno_edge<RW, false>(line, C.weno_eps);
            up[k] = weno_edge<RW, true>(line, C.weno_eps);
          }
        }
        RP::template from_char<dir>(C, x, um, wm);
        RP::template from_char<dir>(C, x, up, wp);
      } else if constexpr (RW == 3) {
        R nn[2 * M], dd[2 * M], vv[2 * M];
#pragma unroll
        for (int k = 0; k < M; ++k)
          weno5_pair<R>(cell[0][k], cell[1][k], cell[2][k], cell[3][k], cell[4][k], cell[5][k],
                        C.weno_eps, nn[k], dd[k], nn[M + k], dd[M + k]);
        div_many<R, 2 * M>(nn, dd, vv);
#pragma unroll
        for (int k = 0; k < M; ++k) {
          wm[k] = vv[k];
          wp[k] = vv[M + k];
        }
      } else {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          R line[NS];
#pragma unroll
          for (int k6 = 0; k6 < NS; ++k6) line[k6] = cell[k6][k];
          wm[k] = weno_edge<RW, false>(line, C.weno_eps);
          wp[k] = weno_edge<RW, true>(line, C.weno_eps);
        }
      }
#pragma unroll
      for (int k = 0; k < M; ++k) {
        ER[k][e] = wm[k];
        EL[k][e] = wp[k];
      }
      R al[MAS], ar[MAS];
      if (MA > 0) {
        const int hil = (dir == 0) ? G + a - 1 : G + b, hir = (dir == 0) ? G + a : G + b;
        const int hjl = (dir == 0) ? ((ND == 2) ? G + b : 0) : G + a - 1;
        const int hjr = (dir == 0) ? ((ND == 2) ? G + b : 0) : G + a;
#pragma unroll
        for (int k = 0; k < MA; ++k) {
          al[k] = At[k][MA > 0 ? hjl : 0][MA > 0 ? OX + hil : 0];
          ar[k] = At[k][MA > 0 ? hjr : 0][MA > 0 ? OX + hir : 0];
        }
      }
      R W[MW][M], s[MW], am[M], ap[M], x[NC];
      RP::template solve<dir>(C, wm, wp, al, ar, W, s, am, ap, x);
#pragma unroll
      for (int k = 0; k < M; ++k) {
        FM[k][e] = am[k];
        FP[k][e] = ap[k];
      }
      // interfaces 0..n of interior lines count for the Courant number
      const int ga = ((dir == 0) ? c0 : r0) + a, gb = ((dir == 0) ? r0 : c0) + b;
      const int nA = (dir == 0) ? nx : ny, nB = (dir == 0) ? ny : nx;
      if (ga <= nA && gb < nB) {
        R m_ = R(0);
        if (C.capa < 0) {
#pragma unroll
          for (int p = 0; p < MW; ++p) m_ = nanmax(m_, (R)fabs(s[p]));
        } else {
          // a wave's Courant number uses the capacity of the cell it enters
          const int hil = (dir == 0) ? G + a - 1 : G + b, hir = (dir == 0) ? G + a : G + b;
          const int hjl = (dir == 0) ? ((ND == 2) ? G + b : 0) : G + a - 1;
          const int hjr = (dir == 0) ? ((ND == 2) ? G + b : 0) : G + a;
          const R kl = Kt[hjl][hil], kr = Kt[hjr][hir];
#pragma unroll
          for (int p = 0; p < MW; ++p)
            m_ = nanmax(m_, gt0(s[p]) ? ::claw::FM<R>::div(s[p], kr)
                                      : (lt0(s[p]) ? ::claw::FM<R>::div(-s[p], kl) : R(0)));
        }
        if (dir == 0) smx = nanmax(smx, m_);
        else smy = nanmax(smy, m_);
      }
    };
    // the y-interfaces start on a warp boundary of the loop so that no warp
    // runs both directions' code (slots NEX .. NEXP-1 stay idle)
    constexpr int NEXP = (ND == 2) ? (NEX + 31) / 32 * 32 : NEX;
    for (int t = skip ? NEXP + NEY : tid; t < NEXP + NEY; t += NT) {
      if (t < NEX) interface(std::integral_constant<int, 0>{}, t, t);
      else if constexpr (ND == 2) {
        if (t >= NEXP) interface(std::integral_constant<int, 1>{}, t - NEXP, NEX + t - NEXP);
      }
    }
    __syncthreads();

    // (c) the in-cell Riemann problems (q^L_i, q^R_i) and the cell's L, x then y
    auto incell = [&](auto dirc, int ci, int cj) {
      constexpr int dir = decltype(dirc)::value;
      const int na = (dir == 0) ? TX + 1 : TY + 1;
      const int a = (dir == 0) ? ci : cj, b = (dir == 0) ? cj : ci;
      const int e0 = (dir == 0 ? 0 : NEX) + b * na + a, e1 = e0 + 1;
      R ql[M], qr[M], al[MAS];
#pragma unroll
      for (int k = 0; k < M; ++k) {
        ql[k] = EL[k][e0];
        qr[k] = ER[k][e1];
      }
      if (MA > 0) {
#pragma unroll
        for (int k = 0; k < MA; ++k)
          al[k] = At[k][MA > 0 ? ((ND == 2) ? G + cj : 0) : 0][MA > 0 ? OX + G + ci : 0];
      }
      // total fluctuation A dQ_i = A^- + A^+ of the solve (q^L_i, q^R_i), which
      // for every conservative solver here equals the flux jump
      // f(q^R_i) - f(q^L_i); systems with a non-conservative component
      // (the advected tracer) take the solve itself
      R adq[M];
      if constexpr (incell_solve<RP>::value) {
        R W[MW][M], s_[MW], am[M], ap[M], x[NC];
        RP::template solve<dir>(C, ql, qr, al, al, W, s_, am, ap, x);
#pragma unroll
        for (int k = 0; k < M; ++k) adq[k] = am[k] + ap[k];
      } else {
        R fl[M], fr[M];
        RP::template flux<dir>(C, ql, al, fl);
        RP::template flux<dir>(C, qr, al, fr);
#pragma unroll
        for (int k = 0; k < M; ++k) adq[k] = fr[k] - fl[k];
      }
      // with a capacity the cell's L is -(1/(kappa_i dx)) (...)
      const R idn = s_idn[dir];
      const R idk = C.capa < 0 ? idn
                               : ::claw::FM<R>::div(idn, Kt[(ND == 2) ? G + cj : 0][G + ci]);
#pragma unroll
      for (int k = 0; k < M; ++k) L[k] -= (FP[k][e0] + FM[k][e1] + adq[k]) * idk;
    };
    // thread cidx == tid owns cell (ci, cj) (NT == TX*TY)
    for (int cidx = skip ? TX * TY : tid; cidx < TX * TY; cidx += NT) {
      const int ci = cidx % TX, cj = cidx / TX;
      incell(std::integral_constant<int, 0>{}, ci, cj);
      if constexpr (ND == 2) incell(std::integral_constant<int, 1>{}, ci, cj);
    }
    // (no barrier: the combination below reads only this thread's L and the
    // staged Q^(k); the barriers of finish_attempt precede the next tile)

    // (d) Runge-Kutta stage combination: v = Q^(k) + g dt L, then up to two
    // linear combinations with earlier states
    if (!skip) {
      const int c = c0 + ti, r = r0 + tj;
      if (c < nx && r < ny) {
        const size_t off = (size_t)r * nx + c;
        const R gdt = (R)op.g * s_dt;
        const R a0 = (R)op.a0, a1 = (R)op.a1, b0 = (R)op.b0, b1 = (R)op.b1;
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const R qkv = Qt[k][(ND == 2) ? G + tj : 0][OX + G + ti];
          const R v = qkv + gdt * L[k];
          const R o = (op.a0 != 0.0) ? a0 * qa[k * plane + off] + a1 * v : a1 * v;
          bad |= !isfinite(o);
          qo[k * plane + off] = o;
          if (qo2) {
            const R o2 = (op.b0 != 0.0) ? b0 * qb[k * plane + off] + b1 * v : b1 * v;
            qo2[k * plane + off] = o2;
          }
        }
      }
    }
    finish_attempt<R>(ctl, smx, smy, bad, mb.ntiles, op.last != 0);
  }
}

}  // namespace claw
