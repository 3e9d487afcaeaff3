// classic.cuh -- fused Clawpack-classic step kernels.
//
// One launch = one attempt of one step for every member of a tile table:
// ghost-cell remap in the loads, Riemann solve at every interface, wave
// limiting, second-order corrections (Eq. (lwflux)), transverse corrections in
// 2D (Sec. 2.1; LeVeque 1997), conservative update (Eq. (fluxdiff)) and the
// maximum wave speed.  In 2D the last block of a member to finish runs the
// CFL controller (Sec. 4); in 1D each warp folds its speed into the control
// block by atomics and either the warp whose item completes the member's
// attempt (single-unit items) or a controller launch after the kernel (whole
// tiles) runs the controller.
#pragma once

#include "async_copy.cuh"
#include "kernels.h"
#include "riemann.cuh"

namespace claw {

// ---------------------------------------------------------------------------
// 1D: each lane owns K consecutive cells, loaded with 16-byte vector loads
// when the fields are aligned (ghost cells by index remap).  It prepares its
// cells once (CellPrep: the per-cell part of the Riemann solve) and solves the
// K interfaces on their left, the first one with the prepared cell of the
// lane below (a warp shuffle).  Limiting interface k needs the waves of
// interfaces k-1 and k+1, and the update of the last cell needs the
// fluctuation and correction of interface K: those come from the neighbour
// lanes by shuffles too.  Lanes 0 and 31 are the warp's halo and write
// nothing, so a warp writes 30 K cells and no cell is prepared or solved
// twice inside it.  No block barrier: each warp reads its member's control
// values itself.  With single-unit work items the warp whose item completes a
// member's attempt (an arrival count per member) runs that member's
// controller; with whole tiles a controller launch follows the kernel.
// ---------------------------------------------------------------------------
// cache hint: fetch the 128-byte line holding p into L1 (no register
// result; p must lie inside an allocation)
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

template <typename R, int K>
struct VecIO;
template <>
struct VecIO<float, 4> {
  // from a 16-byte aligned shared-memory slot
  __device__ static __forceinline__ void load_shared(const float* p, float (&v)[4]) {
    const float4 a = *(const float4*)p;
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  __device__ static __forceinline__ void load(const float* p, float (&v)[4]) {
    const float4 a = __ldg((const float4*)p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  __device__ static __forceinline__ void store(float* p, const float (&v)[4]) {
    ((float4*)p)[0] = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct VecIO<float, 8> {
  // from a 16-byte aligned shared-memory slot
  __device__ static __forceinline__ void load_shared(const float* p, float (&v)[8]) {
    const float4 a = ((const float4*)p)[0], b = ((const float4*)p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
  __device__ static __forceinline__ void load(const float* p, float (&v)[8]) {
    const float4 a = __ldg((const float4*)p), b = __ldg((const float4*)p + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
  __device__ static __forceinline__ void store(float* p, const float (&v)[8]) {
    ((float4*)p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    ((float4*)p)[1] = make_float4(v[4], v[5], v[6], v[7]);
  }
};
template <>
struct VecIO<double, 2> {
  // from a 16-byte aligned shared-memory slot
  __device__ static __forceinline__ void load_shared(const double* p, double (&v)[2]) {
    const double2 a = *(const double2*)p;
    v[0] = a.x; v[1] = a.y;
  }
  __device__ static __forceinline__ void load(const double* p, double (&v)[2]) {
    const double2 a = __ldg((const double2*)p);
    v[0] = a.x; v[1] = a.y;
  }
  __device__ static __forceinline__ void store(double* p, const double (&v)[2]) {
    ((double2*)p)[0] = make_double2(v[0], v[1]);
  }
};
template <>
struct VecIO<double, 4> {
  // from a 16-byte aligned shared-memory slot
  __device__ static __forceinline__ void load_shared(const double* p, double (&v)[4]) {
    const double2 a = ((const double2*)p)[0], b = ((const double2*)p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  __device__ static __forceinline__ void load(const double* p, double (&v)[4]) {
    const double2 a = __ldg((const double2*)p), b = __ldg((const double2*)p + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  __device__ static __forceinline__ void store(double* p, const double (&v)[4]) {
    ((double2*)p)[0] = make_double2(v[0], v[1]);
    ((double2*)p)[1] = make_double2(v[2], v[3]);
  }
};

// Per-cell preparation of a Riemann solve.  The default keeps the raw state
// and aux; solvers with a cell-local part (RpElasticity: exp, sqrt and 1/rho)
// specialise it so that each cell is prepared once instead of once per side.
template <class RP, typename R>
struct CellPrep {
  static constexpr int MAS = RP::MA > 0 ? RP::MA : 1;
  struct Cell {
    R q[RP::M];
    R a[MAS];
  };
  __device__ static __forceinline__ void prep(const MConsts<R>&, const R (&q)[RP::M],
                                              const R (&a)[MAS], Cell& c) {
#pragma unroll
    for (int k = 0; k < RP::M; ++k) c.q[k] = q[k];
#pragma unroll
    for (int k = 0; k < MAS; ++k) c.a[k] = a[k];
  }
  __device__ static __forceinline__ void solve(const MConsts<R>& C, const Cell& l, const Cell& r,
                                               R (&W)[RP::MW][RP::M], R (&s)[RP::MW],
                                               R (&am)[RP::M], R (&ap)[RP::M]) {
    R x[RP::NCTX];
    RP::template solve<0>(C, l.q, r.q, l.a, r.a, W, s, am, ap, x);
  }
};

template <typename R, int ND>
struct RpElasticity;

template <typename R>
struct CellPrep<RpElasticity<R, 1>, R> {
  static constexpr int MAS = 2;
  struct Cell {
    R e;   // exp(K eps) = sigma + 1
    R u;   // m / rho
    R c;   // sqrt(K exp(K eps) / rho)
    R Z;   // rho c
  };
  __device__ static __forceinline__ void prep(const MConsts<R>&, const R (&q)[2],
                                              const R (&a)[2], Cell& c) {
    c.e = FM<R>::exp(a[1] * q[0]);
    if constexpr (sizeof(R) == 4) {
      // one reciprocal square root r = 1/sqrt(K e rho) gives them all:
      // c = K e r, Z = rho c = K e rho r, 1/rho = c r
      const R t = a[1] * c.e;
      const R u = t * a[0];
      const R r = FM<R>::rsqrt(u);
      c.c = t * r;
      c.Z = u * r;
      c.u = q[1] * (c.c * r);
    } else {
      const R ir = FM<R>::rcp(a[0]);
      c.u = q[1] * ir;
      c.c = FM<R>::sqrt(a[1] * c.e * ir);
      c.Z = a[0] * c.c;
    }
  }
  // the f-wave solve of RpElasticity on prepared cells
  __device__ static __forceinline__ void solve(const MConsts<R>&, const Cell& l, const Cell& r,
                                               R (&W)[2][2], R (&s)[2], R (&am)[2], R (&ap)[2]) {
    const R d1 = l.u - r.u;  // jump of -u
    const R d2 = l.e - r.e;  // jump of -sigma
    const R iz = FM<R>::rcp(l.Z + r.Z);
    const R b1 = (r.Z * d1 + d2) * iz;
    const R b2 = (l.Z * d1 - d2) * iz;
    W[0][0] = b1;
    W[0][1] = b1 * l.Z;
    W[1][0] = b2;
    W[1][1] = -b2 * r.Z;
    s[0] = -l.c;
    s[1] = r.c;
    // speeds are -c_l < 0 < c_r: A^-dQ = Z^1, A^+dQ = Z^2
    am[0] = b1;
    am[1] = W[0][1];
    ap[0] = b2;
    ap[1] = W[1][1];
  }
};

// limited second-order correction F (Eq. (lwflux)) of interface `c` from the
// waves of its neighbours `l` and `r` (the upwind one per wave decides theta)
template <class RP, typename R, int LIMC = -1>
__device__ __forceinline__ void limit1d(const MConsts<R>& C, int order,
                                        const R (&Wl)[RP::MW][RP::M],
                                        const R (&Wc)[RP::MW][RP::M], const R (&sc)[RP::MW],
                                        const R (&Wr)[RP::MW][RP::M], R dtdx, R (&F)[RP::M]) {
  constexpr int M = RP::M, MW = RP::MW;
  if (order != 2) {
#pragma unroll
    for (int k = 0; k < M; ++k) F[k] = R(0);
    return;
  }
  R dot[MW], nrm[MW];
  constexpr int KS = strength_k<RP, 0>();
#pragma unroll
  for (int p = 0; p < MW; ++p) {
    // upwind neighbour: left for a right-going wave
    const bool right = signed_waves<RP>::value ? p != 0 : sc[p] > R(0);
    if constexpr (KS >= 0) {
      dot[p] = right ? Wl[p][KS] : Wr[p][KS];
      nrm[p] = Wc[p][KS];
    } else {
      R d = R(0), n2 = R(0);
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const R up = right ? Wl[p][k] : Wr[p][k];
        d += up * Wc[p][k];
        n2 += Wc[p][k] * Wc[p][k];
      }
      dot[p] = d;
      nrm[p] = n2;
    }
  }
  correction<RP, R, 0, LIMC>(C, Wc, sc, dot, nrm, dtdx, F);
}

// Shared-memory ring of the staged form: per warp S slots, each holding the
// 32 K cells of every field (and aux field) that one warp unit reads, and one
// barrier per slot.
template <typename R, int NW, int S, int NF, int FOOT>
struct Ring1d {
  alignas(128) R cell[NW][S][NF][FOOT];
  alignas(8) unsigned long long bar[NW][S];
};
template <typename R, int NW, int NF, int FOOT>
struct Ring1d<R, NW, 0, NF, FOOT> {};

// FAST: the MC limiter and second order fixed at compile time (the launcher
// takes it for FP32 methods with those settings).
// S > 0 (staged form): a unit whose 32 K cells lie inside the grid, with
// 16-byte aligned fields, arrives in shared memory by bulk asynchronous
// copies (one per field) that the warp's lane 0 issues up to S units ahead,
// into a ring of S slots; the lanes read their cells from the slot.  Edge
// units and unaligned fields take the direct loads.  The arithmetic is the
// same either way, so both forms give the same bits.
template <class RP, typename R, int NT, int K, int SPW, bool FAST = false, int S = 0>
__global__ void __launch_bounds__(NT, (sizeof(R) == 4 && RP::M <= 2) ? (K >= 8 ? 4 : 8) : 1)
    classic1d_kernel(const Member* __restrict__ members, const Tile* __restrict__ tiles,
                     int ntiles_total, const MConsts<R> C) {
  constexpr int M = RP::M, MW = RP::MW, MA = RP::MA;
  constexpr int LIMC = FAST ? CLAW_LIM_MC : -1;
  const int order = FAST ? 2 : C.order;
  constexpr int MAS = MA > 0 ? MA : 1;
  constexpr int NW = NT / 32;      // warp units per tile
  constexpr int WC = 30 * K;       // cells a warp unit writes (lanes 1..30)
  // the halo lane 0 solves interfaces between its own cells only: with K >= 2
  // its last one is the valid left neighbour that lane 1's limiter needs
  static_assert(K >= 2, "two or more cells per lane");
  constexpr int T = NW * WC;       // cells per tile
  constexpr unsigned FULL = 0xffffffffu;
  using CP = CellPrep<RP, R>;
  using Cell = typename CP::Cell;
  constexpr int NCR = sizeof(Cell) / sizeof(R);
  static_assert(NCR * sizeof(R) == sizeof(Cell), "Cell holds values of type R only");
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;  // warp in block
  // Launched as a programmatic dependent of the previous attempt (single-unit
  // launches of small grids): wait until that launch has completed and its
  // memory is visible, then let the next attempt's launch begin (its blocks
  // wait here in turn), so that launch latency overlaps this attempt.  For a
  // launch without the attribute both return at once.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  // staged form: the ring, and the warp's producer cursor (the consumer's
  // sequence of units, walked up to S units ahead)
  constexpr int NF = M + MA;    // fields a unit reads
  constexpr int FOOT = 32 * K;  // cells of a unit's footprint (lanes 0..31)
  static_assert(S == 0 || (FOOT * sizeof(R)) % 16 == 0, "bulk copies move multiples of 16 B");
  __shared__ Ring1d<R, NW, S, NF, FOOT> ring;
  bool failed = false;                   // a bounded wait of this warp gave up
  [[maybe_unused]] unsigned phase = 0u;  // expected parity per slot
  [[maybe_unused]] unsigned pend = 0u;   // slots with a copy in flight
  [[maybe_unused]] int j = 0, pj = 0;    // units consumed; units the producer passed
  // producer cursor: item p_it; its unit starting at cell p_us (valid while
  // p_us < p_uend, the end of the item's units in the grid); p_q, p_a the
  // item's input fields, p_q null when they cannot be copied in bulk
  [[maybe_unused]] int p_it = 0, p_us = 0, p_uend = 0, p_nx = 0;
  [[maybe_unused]] const R* p_q = nullptr;
  [[maybe_unused]] const R* p_a = nullptr;
  // fields that bulk copies may read: 16-byte aligned bases and rows
  auto stage_ok = [&](const R* qq, const R* aa, int n) {
    const bool rows16 = ((size_t)n * sizeof(R)) % 16 == 0;
    return ((size_t)qq & 15) == 0 && (M == 1 || rows16) &&
           (MA == 0 || (((size_t)aa & 15) == 0 && (MA == 1 || rows16)));
  };
  // a unit whose whole footprint [ustart - K, ustart + 31 K) lies in the grid
  auto stage_unit = [&](int ustart, int n) { return ustart >= K && ustart + 31 * K <= n; };
  // move the producer cursor to the next item with a unit in the grid
  auto p_next_item = [&]() {
    for (;;) {
      p_it += gridDim.x * NW;
      if (p_it >= ntiles_total * (NW / SPW)) {
        p_us = p_uend = 0;
        return;
      }
      const Tile tl = tiles ? tiles[p_it / (NW / SPW)] : Tile{0, p_it / (NW / SPW)};
      const Member& mb = members[tl.member];
      const DevCtl* pc = mb.ctl;
      if (pc->done) continue;
      p_nx = mb.nx;
      p_us = tl.tile * T + (p_it % (NW / SPW)) * SPW * WC;
      p_uend = min(p_nx, p_us + SPW * WC);
      if (p_us >= p_uend) continue;
      p_q = (const R*)mb.q[pc->cur];
      p_a = (const R*)mb.aux;
      if (!stage_ok(p_q, p_a, p_nx)) p_q = nullptr;
      return;
    }
  };
  // the producer's unit into slot pj % S (lane 0 issues), then the next one.
  // The slot was last read at the start of unit pj - S, whose cell values
  // every lane has since used in arithmetic and passed through full-warp
  // shuffles, so those reads are complete before lane 0 refills the slot.
  auto p_issue = [&]() {
    if constexpr (S > 0) {
      const int slot = pj % S;
      if (p_q && stage_unit(p_us, p_nx)) {
        if (lane == 0) {
          const unsigned bar = smem_u32(&ring.bar[wib][slot]);
          constexpr unsigned fb = FOOT * sizeof(R);
          mbar_arrive_expect_tx(bar, NF * fb);
#pragma unroll
          for (int f = 0; f < M; ++f)
            bulk_g2s(smem_u32(&ring.cell[wib][slot][f][0]), p_q + (size_t)f * p_nx + p_us - K,
                     fb, bar);
#pragma unroll
          for (int f = 0; f < MA; ++f)
            bulk_g2s(smem_u32(&ring.cell[wib][slot][M + f][0]),
                     p_a + (size_t)f * p_nx + p_us - K, fb, bar);
        }
        pend |= 1u << slot;
      }
      ++pj;
      p_us += WC;
      if (p_us >= p_uend) p_next_item();
    }
  };
  if constexpr (S > 0) {
    if (lane == 0) {
#pragma unroll
      for (int sl = 0; sl < S; ++sl) mbar_init(smem_u32(&ring.bar[wib][sl]), 1u);
      fence_mbar_init();
    }
    __syncwarp();
    p_it = blockIdx.x * NW + wib - gridDim.x * NW;
    p_next_item();
  }

  // A warp takes a work item: SPW consecutive units of one tile (SPW = NW,
  // or 1 when the tiles are too few to give every resident warp an item).  It
  // reads the member and control values once per item, asks L1 for each next
  // unit's cells while it works on the current one, and folds its speeds into
  // the control block once per item.  No block barrier: the warps of a block
  // overlap one another's loads, arithmetic and stores.
  constexpr int spw = SPW;
  static_assert(NW % SPW == 0, "an item is a whole number of a tile's units");
  constexpr int ipt = NW / spw;  // items per tile
  const int nitems = ntiles_total * ipt;
  for (int it = blockIdx.x * NW + (threadIdx.x >> 5); it < nitems; it += gridDim.x * NW) {
    const Tile tl = tiles ? tiles[it / ipt] : Tile{0, it / ipt};
    const Member& mb = members[tl.member];
    DevCtl* ctl = mb.ctl;
    if (ctl->done) continue;  // uniform over the warp
    const int nx = mb.nx;
    const int sub0 = (it % ipt) * spw;
    const int t0 = tl.tile * T;
    if (t0 + sub0 * WC >= nx) continue;
    const int cur = ctl->cur, nbuf = ctl->nbuf;
    // FP32: one multiply by the stored 1/dx; FP64: the exact quotient
    R dtdx;
    if constexpr (sizeof(R) == 4) dtdx = (R)(ctl->dt * ctl->idx[0]);
    else dtdx = ctl->dt / ctl->dx[0];
    const R* __restrict__ q = (const R*)mb.q[cur];
    R* __restrict__ qo = (R*)mb.q[(cur + 1) % nbuf];
    const R* __restrict__ aux = (const R*)mb.aux;
    const bool rows16 = ((size_t)nx * sizeof(R)) % 16 == 0;  // every field 16-B aligned
    const bool q_ok = ((((size_t)q) | ((size_t)qo)) & 15) == 0 && (M == 1 || rows16);
    const bool a_ok = MA == 0 || ((((size_t)aux) & 15) == 0 && (MA == 1 || rows16));
    [[maybe_unused]] const bool s_ok = S > 0 && stage_ok(q, aux, nx);  // as p_q != null
    R smax = R(0);
    int bad = 0;
    float nf = 0.f;  // FP32: sum of result * 0
    for (int sub = sub0; sub < sub0 + spw; ++sub) {
      const int ustart = t0 + sub * WC;
      if (ustart >= nx || failed) break;  // uniform over the warp

      // lane l holds cells g0 .. g0+K-1; lanes 0 and 31 are the unit's halo
      const int g0 = ustart + (lane - 1) * K;
      if constexpr (S > 0) {
        // keep the producer S units ahead (the slot it refills was read by
        // the previous unit)
        while (!failed && p_us < p_uend && pj < j + S) p_issue();
      } else if (sub + 1 < sub0 + spw) {
        // L1 prefetch of this lane's cells of the next unit
        const int gn = g0 + WC;
        if (gn >= 0 && gn < nx) {
#pragma unroll
          for (int f = 0; f < M + MA; ++f)
            prefetch_l1(f < M ? (const void*)(q + (size_t)f * nx + gn)
                              : (const void*)(aux + (size_t)(f - M) * nx + gn));
        }
      }
      const bool inside = g0 >= 0 && g0 + K <= nx;
      const bool vec = inside && q_ok && a_ok;
      R qa[K][M];
      R aa[K][MAS];
      bool staged = false;
      if constexpr (S > 0) staged = s_ok && stage_unit(ustart, nx);
      if (staged) {
        if constexpr (S > 0) {
          const int slot = j % S;
          const unsigned bit = 1u << slot;
          bool got = mbar_wait_bounded(smem_u32(&ring.bar[wib][slot]), (phase & bit) ? 1u : 0u);
          got = __all_sync(FULL, got);
          if (!got) {
            // a copy that did not complete in time: wait (bounded) for the
            // copies still in flight, report it, and compute nothing more
            // (the warp still arrives for its items, so the controller runs)
#pragma unroll
            for (int sl = 0; sl < S; ++sl)
              if ((pend >> sl) & 1u)
                mbar_wait_bounded(smem_u32(&ring.bar[wib][sl]), (phase >> sl) & 1u);
            failed = true;
            bad |= 2;
            break;
          }
          phase ^= bit;
          pend &= ~bit;
#pragma unroll
          for (int k = 0; k < M; ++k) {
            R v[K];
            VecIO<R, K>::load_shared(&ring.cell[wib][slot][k][lane * K], v);
#pragma unroll
            for (int c = 0; c < K; ++c) qa[c][k] = v[c];
          }
#pragma unroll
          for (int k = 0; k < MA; ++k) {
            R v[K];
            VecIO<R, K>::load_shared(&ring.cell[wib][slot][M + k][lane * K], v);
#pragma unroll
            for (int c = 0; c < K; ++c) aa[c][k] = v[c];
          }
        }
      } else if (vec) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          R v[K];
          VecIO<R, K>::load(q + (size_t)k * nx + g0, v);
#pragma unroll
          for (int c = 0; c < K; ++c) qa[c][k] = v[c];
        }
#pragma unroll
        for (int k = 0; k < MA; ++k) {
          R v[K];
          VecIO<R, K>::load(aux + (size_t)k * nx + g0, v);
#pragma unroll
          for (int c = 0; c < K; ++c) aa[c][k] = v[c];
        }
      } else if (inside) {
        // interior cells of fields that are not 16-byte aligned (rows whose
        // length is not a multiple of the vector): plain loads, no remap
#pragma unroll
        for (int c = 0; c < K; ++c) {
#pragma unroll
          for (int k = 0; k < M; ++k) qa[c][k] = __ldg(q + (size_t)k * nx + g0 + c);
#pragma unroll
          for (int k = 0; k < MA; ++k) aa[c][k] = __ldg(aux + (size_t)k * nx + g0 + c);
        }
      } else {
        // ghost cells by remap; cells beyond the two-cell ghost layer are
        // clamped into it (only halo lanes hold them and nothing reads them)
#pragma unroll
        for (int c = 0; c < K; ++c) {
          const int gi = max(-2, min(g0 + c, nx + 1));
          load_cell<M, R>(C, q, nx, 1, gi, 0, RP::WALL_X, -1, qa[c]);
          if (MA > 0) load_aux<MA, R>(C, aux, nx, 1, gi, 0, aa[c]);
        }
      }

      // each cell prepared once; interface k lies between cells k-1 and k
      // (global index g0+k), its left cell from the lane below
      Cell pc[K];
#pragma unroll
      for (int c = 0; c < K; ++c) CP::prep(C, qa[c], aa[c], pc[c]);
      Cell left;
      {
        const R* a = reinterpret_cast<const R*>(&pc[K - 1]);
        R* b = reinterpret_cast<R*>(&left);
#pragma unroll
        for (int i = 0; i < NCR; ++i) b[i] = __shfl_up_sync(FULL, a[i], 1);
      }
      R W[K][MW][M], s[K][MW], am[K][M], ap[K][M];
      CP::solve(C, left, pc[0], W[0], s[0], am[0], ap[0]);
#pragma unroll
      for (int k = 1; k < K; ++k) CP::solve(C, pc[k - 1], pc[k], W[k], s[k], am[k], ap[k]);

      // max speed over the unit's interfaces ustart .. ustart+WC that are
      // <= nx: lanes 1..30 their K, lane 31 its first, lane 0 none
      const int nsp = min(lane == 0 ? 0 : (lane == 31 ? 1 : K), nx + 1 - g0);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (k < nsp) {
#pragma unroll
          for (int p = 0; p < MW; ++p) {
            // FP32: a non-finite speed makes the results non-finite too, and
            // the finiteness sum below reports those, so a plain max will do
            if constexpr (sizeof(R) == 4) smax = fmaxf(smax, fabsf(s[k][p]));
            else smax = nanmax(smax, (R)fabs(s[k][p]));
          }
        }
      }

      // waves of interface -1 (lane below) and K (lane above)
      R Wm[MW][M], Wp[MW][M], sp[MW], amK[M];
#pragma unroll
      for (int p = 0; p < MW; ++p) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          Wm[p][k] = __shfl_up_sync(FULL, W[K - 1][p][k], 1);
          Wp[p][k] = __shfl_down_sync(FULL, W[0][p][k], 1);
        }
        sp[p] = __shfl_down_sync(FULL, s[0][p], 1);
      }
#pragma unroll
      for (int k = 0; k < M; ++k) amK[k] = __shfl_down_sync(FULL, am[0][k], 1);

      // limit interfaces 0..K-1 (F of interface K comes from the lane above)
      // and update each cell once both of its interfaces are limited:
      // Q_c - dt/dx [(A+dQ - F)_{c-1/2} + (A-dQ + F)_{c+1/2}]
      R qout[K][M], Fl[M], FK[M];
      limit1d<RP, R, LIMC>(C, order, Wm, W[0], s[0], K > 1 ? W[1] : Wp, dtdx, Fl);
#pragma unroll
      for (int k = 0; k < M; ++k) FK[k] = __shfl_down_sync(FULL, Fl[k], 1);
#pragma unroll
      for (int c = 1; c < K; ++c) {
        R Fr[M];
        limit1d<RP, R, LIMC>(C, order, W[c - 1], W[c], s[c], c + 1 < K ? W[c + 1] : Wp, dtdx, Fr);
#pragma unroll
        for (int k = 0; k < M; ++k) {
          qout[c - 1][k] = qa[c - 1][k] - dtdx * ((ap[c - 1][k] - Fl[k]) + (am[c][k] + Fr[k]));
          Fl[k] = Fr[k];
        }
      }
#pragma unroll
      for (int k = 0; k < M; ++k)
        qout[K - 1][k] = qa[K - 1][k] - dtdx * ((ap[K - 1][k] - Fl[k]) + (amK[k] + FK[k]));

      // non-finite results: FP32 folds them into one sum of v * 0 (NaN for
      // a NaN or an infinity, else 0) tested once per item; FP64 tests each
      // value on its bit pattern (the FP64 pipe is the scarce unit)
      if (lane >= 1 && lane <= 30) {
        if (vec && g0 + K <= ustart + WC) {
#pragma unroll
          for (int k = 0; k < M; ++k) {
            R v[K];
#pragma unroll
            for (int c = 0; c < K; ++c) {
              v[c] = qout[c][k];
              if constexpr (sizeof(R) == 4) nf = fmaf(v[c], 0.f, nf);
              else bad |= !isfinite(v[c]);
            }
            VecIO<R, K>::store(qo + (size_t)k * nx + g0, v);
          }
        } else if (inside) {
          // unaligned rows: plain stores of the lane's interior cells
#pragma unroll
          for (int k = 0; k < M; ++k) {
#pragma unroll
            for (int c = 0; c < K; ++c) {
              if constexpr (sizeof(R) == 4) nf = fmaf(qout[c][k], 0.f, nf);
              else bad |= !isfinite(qout[c][k]);
              qo[(size_t)k * nx + g0 + c] = qout[c][k];
            }
          }
        } else {
#pragma unroll
          for (int c = 0; c < K; ++c) {
            if (g0 + c < nx) {
#pragma unroll
              for (int k = 0; k < M; ++k) {
                if constexpr (sizeof(R) == 4) nf = fmaf(qout[c][k], 0.f, nf);
                else bad |= !isfinite(qout[c][k]);
                qo[(size_t)k * nx + g0 + c] = qout[c][k];
              }
            }
          }
        }
      }
      if constexpr (S > 0) ++j;
    }  // units of the item
    if constexpr (sizeof(R) == 4) bad |= !isfinite(nf);
    // per-warp atomics; with single-unit items (the small grids, where a
    // launch more per attempt is felt) the warp that completes the member's
    // attempt runs its controller, with whole tiles (the large grids and
    // batches, where a fence per item would stall the warps) a controller
    // launch follows
    fold_warp<R>(ctl, smax, bad);
    if constexpr (SPW == 1) {
      if (lane == 0) {
        __threadfence();
        const unsigned items = (unsigned)((nx + WC - 1) / WC);
        if (atomicAdd(&ctl->arrive, 1u) == items - 1u) {
          __threadfence();
          run_controller(ctl);
        }
      }
      __syncwarp();
    }
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
// normal solve between two cells, with the solver's per-cell prep when it
// has one (computed once per cell instead of once per interface side)
template <class RP, int DIR, typename R, int NP>
__device__ __forceinline__ void solve_cells(const MConsts<R>& C, const R (&ql)[RP::M],
                                            const R (&qr)[RP::M], const R (&pcl)[NP],
                                            const R (&pcr)[NP], R (&W)[RP::MW][RP::M],
                                            R (&s)[RP::MW], R (&am)[RP::M], R (&ap)[RP::M],
                                            R (&x)[RP::NCTX]) {
  if constexpr (RP::NPC > 0)
    RP::template solve_pc<DIR>(C, ql, qr, pcl, pcr, W, s, am, ap, x);
  else
    RP::template solve<DIR>(C, ql, qr, nullptr, nullptr, W, s, am, ap, x);
}

// sweep: 0 the unsplit step (Q^n in slot 0 -> slot 1, runs the controller);
// dimensional splitting (Godunov) as two launches: 1 the x sweeps (slot 0 ->
// slot 1), 2 the y sweeps (slot 1 -> slot 2, runs the controller).
// FAST: the MC limiter, second order and transverse mode 2 fixed at compile
// time (the launcher takes it for FP32 methods with those settings)
template <class RP, typename R, int BW, bool FAST = false>
__global__ void __launch_bounds__(BW)
    classic2d_kernel(const Member* __restrict__ members, const Tile* __restrict__ tiles,
                     int ntiles_total, const MConsts<R> C, int H, int sweep) {
  constexpr int M = RP::M, MW = RP::MW, NC = RP::NCTX;
  constexpr int LIMC = FAST ? CLAW_LIM_MC : -1;
  const int order = FAST ? 2 : C.order;
  const int transverse = FAST ? 2 : C.transverse;
  constexpr int NP = RP::NPC > 0 ? RP::NPC : 1;
  using NZX = typename RP::template NZ<0>;
  using NZY = typename RP::template NZ<1>;
  // limiter ratios from wave strengths where the solver has them
  constexpr int KSX = strength_k<RP, 0>(), KSY = strength_k<RP, 1>();
  constexpr int TX = BW - 4;
  // neighbour contributions: systems of up to three fields publish the raw
  // vectors (the receiver multiplies and adds them, saving the sender's pass
  // into a zeroed sum); larger systems publish per-row sums (mailboxes)
  constexpr bool GATHER = (M <= 3);
  __shared__ R qs[M][BW];
  __shared__ R pcs[NP][BW];
  __shared__ R xws[MW][M][BW];
  constexpr int MM = GATHER ? 1 : M, BM = GATHER ? 1 : BW;  // mailbox extents
  constexpr int GM = GATHER ? M : 1, BG = GATHER ? BW : 1;  // raw-vector extents
  __shared__ R mbl[4][MM][BM];
  __shared__ R mbr[2][MM][BM];
  __shared__ R gxv[3][GM][BG];  // A^-dQ + F, B^+ and B^- of it (x-interface)
  __shared__ R gyv[4][GM][BG];  // x-splits of the y-fluctuations: A^- (B^+..),
                                // A^- (B^-..), A^+ (B^+..), A^+ (B^-..)
  __shared__ int s_done, s_cur, s_nbuf;
  __shared__ R s_k[3];  // dt/dx, dt/dy, dt^2/(2 dx dy)
  const int l = threadIdx.x;

  for (int it = blockIdx.x; it < ntiles_total; it += gridDim.x) {
    const Tile tl = tiles ? tiles[it] : Tile{0, it};
    const Member& mb = members[tl.member];
    DevCtl* ctl = mb.ctl;
    if (l == 0) {
      s_done = ctl->done;
      const double dtd = ctl->dt;
      s_k[0] = (R)(dtd / ctl->dx[0]);
      s_k[1] = (R)(dtd / ctl->dx[1]);
      s_k[2] = (R)(0.5 * (dtd / ctl->dx[0]) * (dtd / ctl->dx[1]));
      s_cur = ctl->cur;
      s_nbuf = ctl->nbuf;
    }
    __syncthreads();
    if (s_done) {
      __syncthreads();
      continue;
    }
    const int nx = mb.nx, ny = mb.ny;
    const Classic2dLayout L = classic2d_layout(nx, ny, BW, H);
    const int c0 = (tl.tile % L.nsx) * TX;
    const int ch = tl.tile / L.nsx;
    const int r0 = (int)(((long long)ch * ny) / L.nch);
    const int rend = (int)(((long long)(ch + 1) * ny) / L.nch) - 1;
    // a warp whose columns all lie past the second ghost column feeds no
    // stored cell, speed or flag: it only keeps the block's barriers
    const bool live = c0 - 2 + (l & ~31) <= nx + 1;
    const int c = c0 - 2 + l;
    const int cload = min(c, nx + 1);
    const bool col_in = (l >= 2) && (l < BW - 2) && (c < nx);
    const bool xlim = (l >= 2) && (l <= BW - 2);
    const bool xcfl = xlim && (c <= nx);
    const bool ylim = (l >= 1) && (l <= BW - 2);
    const bool dox = sweep != 2, doy = sweep != 1;
    const R* __restrict__ q = (const R*)step_input(mb, s_cur, s_nbuf, sweep == 2 ? 1 : 0);
    R* __restrict__ qo = (R*)mb.q[(s_cur + (sweep == 2 ? 2 : 1)) % s_nbuf];
    const R dtdx = s_k[0], dtdy = s_k[1], kxy = s_k[2];
    const size_t plane = (size_t)nx * ny;

    const ColMap cm = col_map(C, cload, nx);  // the thread's column, remapped once
    R qm2[M], qm1[M], qc[M];
    R pm1[NP], pcc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) pm1[k] = pcc[k] = R(0);
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
    R smx = R(0), smy = R(0);
    int bad = 0;

    for (int Rw = r0 - 2; Rw <= rend + 2; ++Rw) {
      // (1) load row Rw
#pragma unroll
      for (int k = 0; k < M; ++k) {
        qm2[k] = qm1[k];
        qm1[k] = qc[k];
      }
      if (live) {
        load_cell_col<M, R>(C, q, nx, ny, cm, Rw, RP::WALL_X, RP::WALL_Y, qc);
#pragma unroll
        for (int k = 0; k < M; ++k) qs[k][l] = qc[k];
        if constexpr (RP::NPC > 0) {
#pragma unroll
          for (int k = 0; k < NP; ++k) pm1[k] = pcc[k];
          RP::cell_pc(C, qc, pcc);
#pragma unroll
          for (int k = 0; k < NP; ++k) pcs[k][l] = pcc[k];
        }
      }

      // (2) y-interface Rw (rows Rw-1, Rw)
      R nW[MW][M], ns[MW], nam[M], nap[M], nx_[NC], nnrm[MW], ndot[MW];
      const bool yrow = live && doy && Rw >= r0 - 1;
      if (yrow) {
        solve_cells<RP, 1, R, NP>(C, qm1, qc, pm1, pcc, nW, ns, nam, nap, nx_);
#pragma unroll
        for (int p = 0; p < MW; ++p) {
          if constexpr (KSY >= 0) {
            // wave strengths: the new interface's strength serves as its
            // "norm" and as the upper neighbour's term of interface Rw-1
            nnrm[p] = ndot[p] = nW[p][KSY];
          } else {
            R a = R(0), b = R(0);
#pragma unroll
            for (int k = 0; k < M; ++k) {
              if (!NZY::f(p, k)) continue;
              a += nW[p][k] * nW[p][k];
              b += nW[p][k] * yW[p][k];
            }
            nnrm[p] = a;
            ndot[p] = b;
          }
        }
        if (col_in && Rw >= r0 && Rw <= rend + 1) {
#pragma unroll
          for (int p = 0; p < MW; ++p) smy = max_nonneg(smy, (R)fabs(ns[p]));
        }
      }
      __syncthreads();  // qs ready

      // (3) x-interface (c, Rw)
      const bool xrow = live && dox && (Rw >= r0 - 1) && (Rw <= rend + 1);
      R xW[MW][M], xs[MW], xam[M], xap[M], xx[NC];
      if (xrow && l >= 1) {
        R ql[M], pl[NP];
#pragma unroll
        for (int k = 0; k < M; ++k) ql[k] = qs[k][l - 1];
#pragma unroll
        for (int k = 0; k < NP; ++k) pl[k] = RP::NPC > 0 ? pcs[k][l - 1] : R(0);
        solve_cells<RP, 0, R, NP>(C, ql, qc, pl, pcc, xW, xs, xam, xap, xx);
#pragma unroll
        for (int p = 0; p < MW; ++p)
#pragma unroll
          for (int k = 0; k < M; ++k)
            if (NZX::f(p, k)) xws[p][k][l] = xW[p][k];
      }
      __syncthreads();  // x waves ready

      R tl_[4][M], tr_[2][M];
      R gx[3][M], gy[4][M];
#pragma unroll
      for (int k = 0; k < M; ++k) {
        tl_[0][k] = tl_[1][k] = tl_[2][k] = tl_[3][k] = R(0);
        tr_[0][k] = tr_[1][k] = R(0);
        gx[0][k] = gx[1][k] = gx[2][k] = R(0);
        gy[0][k] = gy[1][k] = gy[2][k] = gy[3][k] = R(0);
      }

      // (4) x-limiting, corrections, transverse propagation
      if (xrow && xlim) {
        R F[M];
        if (order == 2) {
          R dot[MW], nrm[MW];
#pragma unroll
          for (int p = 0; p < MW; ++p) {
            const int lu = gt0(xs[p]) ? l - 1 : l + 1;
            if constexpr (KSX >= 0) {
              dot[p] = xws[p][KSX][lu];
              nrm[p] = xW[p][KSX];
            } else {
              R a = R(0), b = R(0);
#pragma unroll
              for (int k = 0; k < M; ++k) {
                if (!NZX::f(p, k)) continue;
                b += xws[p][k][lu] * xW[p][k];
                a += xW[p][k] * xW[p][k];
              }
              dot[p] = b;
              nrm[p] = a;
            }
          }
          correction<RP, R, 0, LIMC>(C, xW, xs, dot, nrm, dtdx, F);
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
          if constexpr (GATHER) gx[0][k] = am_[k];
          else tl_[2][k] -= dtdx * am_[k];
        }
        if (xcfl && Rw >= r0 && Rw <= rend) {
#pragma unroll
          for (int p = 0; p < MW; ++p) smx = max_nonneg(smx, (R)fabs(xs[p]));
        }
        if (transverse) {
          R tp[M], tm[M], bmp[M], bpp[M], bmm[M], bpm[M];
#pragma unroll
          for (int k = 0; k < M; ++k) {
            tp[k] = transverse == 2 ? ap_[k] : xap[k];
            tm[k] = transverse == 2 ? am_[k] : xam[k];
          }
          RP::template trans<0>(C, xx, tp, bmp, bpp);
          RP::template trans<0>(C, xx, tm, bmm, bpm);
#pragma unroll
          for (int k = 0; k < M; ++k) {
            acc2[k] += kxy * (bpp[k] - bmp[k]);
            acc3[k] -= kxy * bpp[k];
            acc1[k] += kxy * bmp[k];
            if constexpr (GATHER) {
              gx[1][k] = bpm[k];
              gx[2][k] = bmm[k];
            } else {
              tl_[2][k] += kxy * (bpm[k] - bmm[k]);
              tl_[3][k] -= kxy * bpm[k];
              tl_[1][k] += kxy * bmm[k];
            }
          }
        }
      }

      // (5) y-limiting of interface Rw-1, corrections, transverse propagation
      if (live && doy && ylim && Rw - 1 >= r0 && Rw - 1 <= rend + 1) {
        R G[M];
        if (order == 2) {
          R dot[MW];
#pragma unroll
          for (int p = 0; p < MW; ++p) dot[p] = gt0(ys[p]) ? ydot[p] : ndot[p];
          correction<RP, R, 1, LIMC>(C, yW, ys, dot, ynrm, dtdy, G);
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
        if (transverse) {
          R tp[M], tm[M], amp[M], app[M], amm[M], apm[M];
#pragma unroll
          for (int k = 0; k < M; ++k) {
            tp[k] = transverse == 2 ? bp_[k] : yap[k];
            tm[k] = transverse == 2 ? bm_[k] : yam[k];
          }
          RP::template trans<1>(C, yx, tp, amp, app);
          RP::template trans<1>(C, yx, tm, amm, apm);
#pragma unroll
          for (int k = 0; k < M; ++k) {
            acc1[k] += kxy * (app[k] - amp[k]);
            acc0[k] += kxy * (apm[k] - amm[k]);
            if constexpr (GATHER) {
              gy[0][k] = amp[k];
              gy[1][k] = amm[k];
              gy[2][k] = app[k];
              gy[3][k] = apm[k];
            } else {
              tr_[1][k] -= kxy * app[k];
              tr_[0][k] -= kxy * apm[k];
              tl_[1][k] += kxy * amp[k];
              tl_[0][k] += kxy * amm[k];
            }
          }
        }
      }
      if (live) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          if constexpr (GATHER) {
            gxv[0][k][l] = gx[0][k];
            gxv[1][k][l] = gx[1][k];
            gxv[2][k][l] = gx[2][k];
            gyv[0][k][l] = gy[0][k];
            gyv[1][k][l] = gy[1][k];
            gyv[2][k][l] = gy[2][k];
            gyv[3][k][l] = gy[3][k];
          } else {
            mbl[0][k][l] = tl_[0][k];
            mbl[1][k][l] = tl_[1][k];
            mbl[2][k][l] = tl_[2][k];
            mbl[3][k][l] = tl_[3][k];
            mbr[0][k][l] = tr_[0][k];
            mbr[1][k][l] = tr_[1][k];
          }
        }
      }
      __syncthreads();  // mailboxes ready

      // (6) gather neighbour contributions, (7) finish row Rw-2
      if (live && l + 1 < BW) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          if constexpr (GATHER) {
            // the right neighbour's x-interface is this column's right face
            const R am_n = gxv[0][k][l + 1], bpm_n = gxv[1][k][l + 1],
                    bmm_n = gxv[2][k][l + 1];
            acc2[k] -= dtdx * am_n;
            acc2[k] += kxy * (bpm_n - bmm_n);
            acc3[k] -= kxy * bpm_n;
            acc1[k] += kxy * bmm_n;
            acc1[k] += kxy * gyv[0][k][l + 1];
            acc0[k] += kxy * gyv[1][k][l + 1];
          } else {
            acc0[k] += mbl[0][k][l + 1];
            acc1[k] += mbl[1][k][l + 1];
            acc2[k] += mbl[2][k][l + 1];
            acc3[k] += mbl[3][k][l + 1];
          }
        }
      }
      if (live && l >= 1) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          if constexpr (GATHER) {
            acc1[k] -= kxy * gyv[2][k][l - 1];
            acc0[k] -= kxy * gyv[3][k][l - 1];
          } else {
            acc0[k] += mbr[0][k][l - 1];
            acc1[k] += mbr[1][k][l - 1];
          }
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
          if constexpr (KSY >= 0) {
            // the lower neighbour's strength of the next interface to limit
            ydot[p] = ynrm[p];
            ynrm[p] = nnrm[p];
          } else {
            ynrm[p] = nnrm[p];
            ydot[p] = ndot[p];
          }
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
    finish_attempt<R>(ctl, smx, smy, bad, mb.ntiles, sweep != 1);
  }
}

}  // namespace claw

