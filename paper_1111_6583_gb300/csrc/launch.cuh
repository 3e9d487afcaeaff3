// launch.cuh -- launchers of the fused kernels for one Riemann solver, and the
// first-order wave-speed kernel used to choose the first dt (Sec. 4).
#pragma once

#include "classic.cuh"
#include "classic3d.cuh"
#include "classic_faces.cuh"
#include "kernels.h"
#include "sharpclaw.cuh"

namespace claw {

// First-order interface solves on the cell averages of every member; block
// maxima of |s| per direction go to ctl->smax (no controller).
template <class RP, typename R, int ND>
__global__ void __launch_bounds__(kMaxspeedCells)
    maxspeed_kernel(const Member* __restrict__ members, const Tile* __restrict__ tiles,
                    int ntiles_total, const MConsts<R> C) {
  constexpr int M = RP::M, MW = RP::MW, MA = RP::MA, MAS = MA > 0 ? MA : 1;
  for (int it = blockIdx.x; it < ntiles_total; it += gridDim.x) {
    const Tile tl = tiles ? tiles[it] : Tile{0, it};
    const Member& mb = members[tl.member];
    DevCtl* ctl = mb.ctl;
    const int nx = mb.nx, ny = (ND == 2) ? mb.ny : 1;
    const long long cell = (long long)tl.tile * kMaxspeedCells + threadIdx.x;
    const R* q = (const R*)mb.q[ctl->cur];
    const R* aux = (const R*)mb.aux;
    R sx = R(0), sy = R(0);
    if (cell < (long long)nx * ny) {
      const int i = (int)(cell % nx), j = (int)(cell / nx);
      R W[MW][M], s[MW], am[M], ap[M], x[RP::NCTX];
      R a[M], b[M], al[MAS], ar[MAS];
      for (int side = 0; side < (i == nx - 1 ? 2 : 1); ++side) {
        load_cell<M, R>(C, q, nx, ny, i - 1 + side, j, RP::WALL_X, RP::WALL_Y, a);
        load_cell<M, R>(C, q, nx, ny, i + side, j, RP::WALL_X, RP::WALL_Y, b);
        if (MA > 0) {
          load_aux<MA, R>(C, aux, nx, ny, i - 1 + side, j, al);
          load_aux<MA, R>(C, aux, nx, ny, i + side, j, ar);
        }
        RP::template solve<0>(C, a, b, al, ar, W, s, am, ap, x);
        if (C.capa < 0) {
#pragma unroll
          for (int p = 0; p < MW; ++p) sx = nanmax(sx, (R)fabs(s[p]));
        } else {
          const R kl = load_aux_field<R>(C, aux, nx, ny, i - 1 + side, j, C.capa);
          const R kr = load_aux_field<R>(C, aux, nx, ny, i + side, j, C.capa);
#pragma unroll
          for (int p = 0; p < MW; ++p)
            sx = nanmax(sx, gt0(s[p]) ? FM<R>::div(s[p], kr)
                                      : (lt0(s[p]) ? FM<R>::div(-s[p], kl) : R(0)));
        }
      }
      if constexpr (ND == 2) {
        for (int side = 0; side < (j == ny - 1 ? 2 : 1); ++side) {
          load_cell<M, R>(C, q, nx, ny, i, j - 1 + side, RP::WALL_X, RP::WALL_Y, a);
          load_cell<M, R>(C, q, nx, ny, i, j + side, RP::WALL_X, RP::WALL_Y, b);
          if (MA > 0) {
            load_aux<MA, R>(C, aux, nx, ny, i, j - 1 + side, al);
            load_aux<MA, R>(C, aux, nx, ny, i, j + side, ar);
          }
          RP::template solve<1>(C, a, b, al, ar, W, s, am, ap, x);
          if (C.capa < 0) {
#pragma unroll
            for (int p = 0; p < MW; ++p) sy = nanmax(sy, (R)fabs(s[p]));
          } else {
            const R kl = load_aux_field<R>(C, aux, nx, ny, i, j - 1 + side, C.capa);
            const R kr = load_aux_field<R>(C, aux, nx, ny, i, j + side, C.capa);
#pragma unroll
            for (int p = 0; p < MW; ++p)
              sy = nanmax(sy, gt0(s[p]) ? FM<R>::div(s[p], kr)
                                        : (lt0(s[p]) ? FM<R>::div(-s[p], kl) : R(0)));
          }
        }
      }
    }
    finish_attempt<R>(ctl, sx, sy, 0, 0, false);
  }
}

inline int launch_grid(int ntiles) { return ntiles < 1 ? 1 : ntiles; }

// Persistent grid: no more blocks than fit on the GPU at once (SMs x resident
// blocks per SM of this kernel); each block walks the tile table with a
// grid stride.  Queried once per kernel (one instantiation per kernel).
template <auto Kern>
inline int persistent_grid(int threads, int ntiles) {
  static int cap = 0;
  if (cap == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, Kern, threads, 0);
    cap = sms * (per > 0 ? per : 1);
    if (cap < 1) cap = 1;
  }
  return ntiles < 1 ? 1 : (ntiles < cap ? ntiles : cap);
}

// Axisymmetric Euler geometric source (Sec. 7.2) by fractional steps: with
// r = y (cell centre) and v the radial velocity,
// psi(q) = -(1/r) (rho v, rho u v, rho v^2, (E + p) v, 0 for a tracer), over a
// time h by the two-stage Runge-Kutta method q1 = q + h psi(q),
// q <- (q + q1 + h psi(q1)) / 2.  A member whose accepted-step count equals
// its source mark has nothing pending (rejected or skipped attempt).
// psi from the conserved variables with one reciprocal of rho (ir = 1/r is
// the caller's): rho v = q2, rho u v = q1 v, rho v^2 = q2 v.
template <class RP, typename R>
__device__ __forceinline__ void axisym_psi(const MConsts<R>& C, const R (&q)[RP::M], R ir,
                                           R (&f)[RP::M]) {
  const R irho = R(1) / q[0];
  const R v = q[2] * irho;
  const R p = C.gm1 * (q[3] - R(0.5) * ((q[1] * q[1] + q[2] * q[2]) * irho));
#pragma unroll
  for (int k = 0; k < RP::M; ++k) f[k] = R(0);
  f[0] = -(q[2] * ir);
  f[1] = -((q[1] * v) * ir);
  f[2] = -((q[2] * v) * ir);
  f[3] = -(((q[3] + p) * v) * ir);
}

// The source ODE over one fractional step by Heun's method, cell by cell.
// phase 0 (Godunov): dt_used in place on the new slot cur, after an accepted
// step only; phase 1 (Strang, before the step): dt/2 of the attempt from slot
// cur into Member::qpre, which the step then reads; phase 2 (Strang, after):
// dt_used/2 in place on the new slot cur, after an accepted step only.
template <class RP, typename R>
__global__ void __launch_bounds__(kMaxspeedCells)
    axisym_source_kernel(const Member* __restrict__ members, const Tile* __restrict__ tiles,
                         int ntiles_total, const MConsts<R> C, int phase) {
  constexpr int M = RP::M;
  for (int it = blockIdx.x; it < ntiles_total; it += gridDim.x) {
    const Tile tl = tiles ? tiles[it] : Tile{0, it};
    const Member& mb = members[tl.member];
    const DevCtl* ctl = mb.ctl;
    if (phase == 1 ? (ctl->done != 0) : (ctl->steps == ctl->src_mark)) continue;
    const int nx = mb.nx, ny = mb.ny;
    const long long cell = (long long)tl.tile * kMaxspeedCells + threadIdx.x;
    if (cell >= (long long)nx * ny) continue;
    const int j = (int)(cell / nx);
    const R* qi = (const R*)mb.q[ctl->cur];
    R* qo = phase == 1 ? (R*)mb.qpre : (R*)mb.q[ctl->cur];
    const size_t plane = (size_t)nx * ny;
    const R dt = (R)(phase == 1 ? 0.5 * ctl->dt : (phase == 2 ? 0.5 * ctl->dt_used : ctl->dt_used));
    const R ir = R(1) / (R)(ctl->lo[1] + ((double)j + 0.5) * ctl->dx[1]);
    R q0[M], q1[M], f0[M], f1[M];
#pragma unroll
    for (int k = 0; k < M; ++k) q0[k] = qi[k * plane + cell];
    axisym_psi<RP, R>(C, q0, ir, f0);
#pragma unroll
    for (int k = 0; k < M; ++k) q1[k] = q0[k] + dt * f0[k];
    axisym_psi<RP, R>(C, q1, ir, f1);
#pragma unroll
    for (int k = 0; k < M; ++k) qo[k * plane + cell] = R(0.5) * (q0[k] + (q1[k] + dt * f1[k]));
  }
}

// static shared memory of classic2d_kernel<RP, R, BW> (its arrays; the block
// reduction adds under 1 KB); a block may declare at most 48 KB statically
template <class RP, typename R>
constexpr size_t classic2d_smem(int bw) {
  // qs, xws, neighbour exchange (mailboxes 6 M or raw vectors 7 M plus the
  // one-row placeholders of the unused form), per-cell prep
  return sizeof(R) * (size_t)bw *
         (size_t)(RP::M + RP::MW * RP::M + (RP::M <= 3 ? 7 : 6) * RP::M +
                  (RP::NPC > 0 ? RP::NPC : 1));
}
template <class RP, typename R>
constexpr bool classic2d_fits(int bw) {
  return classic2d_smem<RP, R>(bw) + 1024 <= 48 * 1024;
}

// the classic step runs on the per-face path with a capacity, and in 2D for
// solvers whose transverse split needs the neighbouring cells' media
template <class RP, int ND>
inline bool uses_faces(int capa) {
  return ND <= 2 && (capa >= 0 || (ND == 2 && trans_aux_rp<RP>::value));
}

template <class RP, typename R, int ND>
struct Launchers {
  static cudaError_t classic(const LaunchArgs& a) {
    const MConsts<R>& C = *(const MConsts<R>*)a.consts;
    if constexpr (ND <= 2) {
      if (uses_faces<RP, ND>(C.capa)) {
        const int nx = a.n3[0], ny = ND == 2 ? a.n3[1] : 1;
        const size_t fx = faces_sweep_threads(ND, nx, ny, 0), fy = faces_sweep_threads(ND, nx, ny, 1);
        // a.sweep: 0 unsplit; 1 / 2 the x / y sweep of a dimensionally split step
        if (a.sweep != 2)
          faces_sweep<RP, R, 0><<<(unsigned)((fx + kFacesThreads - 1) / kFacesThreads),
                                  kFacesThreads, 0, a.stream>>>(a.members, C, ND, 0);
        if (ND == 2 && a.sweep != 1)
          faces_sweep<RP, R, 1><<<(unsigned)((fy + kFacesThreads - 1) / kFacesThreads),
                                  kFacesThreads, 0, a.stream>>>(a.members, C, ND,
                                                                a.sweep == 2 ? 1 : 0);
        const long long nc = (long long)nx * ny;
        faces_update<RP, R><<<(unsigned)((nc + kFacesThreads - 1) / kFacesThreads),
                              kFacesThreads, 0, a.stream>>>(a.members, C, ND, a.sweep);
        return cudaGetLastError();
      }
    }
    if constexpr (ND == 3) {
      const long long nx = a.n3[0], ny = a.n3[1], nz = a.n3[2];
      // with transverse terms the x sweep writes every record first (no fill)
      if (!C.transverse) {
        cudaError_t e = cudaMemsetAsync(a.work3, 0, a.work3_bytes, a.stream);
        if (e != cudaSuccess) return e;
      }
      // x: lanes along x, a block of kXSweepLines y lines walks a segment of
      // z planes; y, z: one block per patch of lines and segment of cells
      // along the sweep
      constexpr int NW = kXSweepLines, NB = sizeof(R) == 4 ? 2 : 1;
      int nxc, nyb, nzs;
      xsweep3d_grid(NW, (int)nx, (int)ny, (int)nz, nxc, nyb, nzs);
      classic3d_xsweep<RP, R, NW, NB><<<(unsigned)(nxc * nyb * nzs), 32 * NW, 0, a.stream>>>(
          a.members, C);
      int npf, nps, nseg;
      sweep3d_grid(1, (int)nx, (int)ny, (int)nz, npf, nps, nseg);
      classic3d_sweep<RP, R, 1><<<(unsigned)(npf * nps * nseg), kPatch3d * kPatch3d, 0,
                                  a.stream>>>(a.members, C);
      sweep3d_grid(2, (int)nx, (int)ny, (int)nz, npf, nps, nseg);
      classic3d_sweep<RP, R, 2><<<(unsigned)(npf * nps * nseg), kPatch3d * kPatch3d, 0,
                                  a.stream>>>(a.members, C);
      classic3d_update<RP, R><<<a.ntiles_total, 256, 0, a.stream>>>(a.members, C);
      return cudaGetLastError();
    } else if constexpr (ND == 2 && RP::MA > 0) {
      // 2D solvers with aux fields have normal solves only (SharpClaw)
      (void)C;
      return cudaErrorNotSupported;
    } else if constexpr (ND == 1) {
      if (sizeof(R) == 4 && C.lim == CLAW_LIM_MC && C.order == 2)
        return classic1d<true>(a, C);
      return classic1d<false>(a, C);
    } else {
      // systems of up to three fields: with more, the two block widths of the
      // fixed-settings form were seen to round differently, and every tile
      // shape must give the same bits
      if (sizeof(R) == 4 && RP::M <= 3 && C.lim == CLAW_LIM_MC && C.order == 2 &&
          C.transverse == 2)
        return classic2d<true>(a, C);
      return classic2d<false>(a, C);
    }
    return cudaGetLastError();
  }
  // FAST (FP32 only): the common settings fixed at compile time
  template <bool FAST>
  static cudaError_t classic1d(const LaunchArgs& a, const MConsts<R>& C) {
    if constexpr (ND == 1 && (!FAST || sizeof(R) == 4)) {
      constexpr int K = classic1d_K(sizeof(R) == 8 ? 0 : 1, RP::MA);
      // a warp takes a whole tile when the tiles fill every resident warp
      // (blocks x NW), else a single unit
      constexpr int NW = kClassic1dThreads / 32;
      constexpr int S = classic1d_S(sizeof(R) == 8 ? 0 : 1, RP::M, RP::MA);
      constexpr auto kt = classic1d_kernel<RP, R, kClassic1dThreads, K, NW, FAST, S>;
      constexpr auto ku = classic1d_kernel<RP, R, kClassic1dThreads, K, 1, FAST, S>;
      const long long cap = (long long)persistent_grid<kt>(kClassic1dThreads, 1 << 30) * NW;
      const bool whole =
          a.h == kWork1dTiles || (a.h != kWork1dUnits && a.ntiles_total >= cap);
      if (whole)
        kt<<<persistent_grid<kt>(kClassic1dThreads, (a.ntiles_total + NW - 1) / NW),
             kClassic1dThreads, 0, a.stream>>>(a.members, a.tiles, a.ntiles_total, C);
      else {
        // single units (small grids, where launch latency is the step's
        // cost): a programmatic dependent launch on the previous attempt
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)persistent_grid<ku>(kClassic1dThreads, a.ntiles_total));
        cfg.blockDim = dim3(kClassic1dThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = a.stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const cudaError_t el = cudaLaunchKernelEx(&cfg, ku, a.members, a.tiles, a.ntiles_total, C);
        if (el != cudaSuccess) return el;
      }
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess || !whole) return e;  // single units run their controllers
      return launch_controllers(a.members, a.nmembers > 0 ? a.nmembers : 1, a.stream);
    } else {
      (void)a;
      (void)C;
      return cudaErrorNotSupported;
    }
  }
  template <bool FAST>
  static cudaError_t classic2d(const LaunchArgs& a, const MConsts<R>& C) {
    if constexpr (ND == 2 && RP::MA == 0 && (!FAST || (sizeof(R) == 4 && RP::M <= 3))) {
      if constexpr (classic2d_fits<RP, R>(128)) {
        if (a.bw == 128) {
          classic2d_kernel<RP, R, 128, FAST><<<launch_grid(a.ntiles_total), 128, 0, a.stream>>>(
              a.members, a.tiles, a.ntiles_total, C, a.h, a.sweep);
          return cudaGetLastError();
        }
      }
      if (a.bw != 64) return cudaErrorInvalidValue;
      classic2d_kernel<RP, R, 64, FAST><<<launch_grid(a.ntiles_total), 64, 0, a.stream>>>(
          a.members, a.tiles, a.ntiles_total, C, a.h, a.sweep);
      return cudaGetLastError();
    } else {
      (void)a;
      (void)C;
      return cudaErrorNotSupported;
    }
  }
  static cudaError_t sharp(const LaunchArgs& a) {
    const MConsts<R>& C = *(const MConsts<R>*)a.consts;
    if constexpr (ND == 3) {
      (void)C;
      return cudaErrorNotSupported;
    } else {
      StageOp op;
      if (a.stage_op) {
        op = *a.stage_op;
      } else {
        const StageOp* rk3;
        stage_table(0, &rk3);
        op = rk3[a.stage];
      }
      cudaError_t e = cudaErrorInvalidValue;
      switch (C.weno_r) {
        case 0:
        case 3: e = sharp_launch<3>(a, C, op); break;
        case 4: e = sharp_launch<4>(a, C, op); break;
        case 5: e = sharp_launch<5>(a, C, op); break;
        case 6: e = sharp_launch<6>(a, C, op); break;
        case 7: e = sharp_launch<7>(a, C, op); break;
        case 8: e = sharp_launch<8>(a, C, op); break;
        case 9: e = sharp_launch<9>(a, C, op); break;
        default: break;
      }
      if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
  }
  // 2D: the tile that (a.bw, a.h) names (sharp2d_shape); the fifth-order
  // stage has every shape of kSharpShapes2 whose static shared memory fits a
  // block, the higher orders the default only (cudaErrorNotSupported
  // otherwise)
  template <int RW>
  static cudaError_t sharp_launch(const LaunchArgs& a, const MConsts<R>& C, const StageOp& op) {
    if constexpr (ND == 1) {
      sharp_stage_kernel<RP, R, 1, kSharpTX1, 1, RW>
          <<<launch_grid(a.ntiles_total), kSharpTX1, 0, a.stream>>>(a.members, a.tiles,
                                                                 a.ntiles_total, C, op);
      return cudaSuccess;
    } else if constexpr (ND == 2) {
      int tx, ty;
      sharp2d_shape(a.bw, a.h, tx, ty);
      if (tx == kSharpTX2 && ty == kSharpTY2) return sharp2d<kSharpTX2, kSharpTY2, RW>(a, C, op);
      if constexpr (RW == 3) {
        if (tx == 32 && ty == 4) return sharp2d<32, 4, RW>(a, C, op);
        if (tx == 32 && ty == 8) return sharp2d<32, 8, RW>(a, C, op);
        if (tx == 16 && ty == 16) return sharp2d<16, 16, RW>(a, C, op);
      }
      return cudaErrorNotSupported;
    } else {
      (void)a;
      (void)C;
      (void)op;
      return cudaErrorNotSupported;
    }
  }
  template <int TX, int TY, int RW>
  static cudaError_t sharp2d(const LaunchArgs& a, const MConsts<R>& C, const StageOp& op) {
    if constexpr (sharp_smem_bytes<RP, R, 2, TX, TY, RW>() <= kSmemPerBlock) {
      sharp_stage_kernel<RP, R, 2, TX, TY, RW>
          <<<launch_grid(a.ntiles_total), TX * TY, 0, a.stream>>>(a.members, a.tiles,
                                                                 a.ntiles_total, C, op);
      return cudaSuccess;
    } else {
      (void)a;
      (void)C;
      (void)op;
      return cudaErrorNotSupported;
    }
  }
  static cudaError_t source(const LaunchArgs& a) {
    const MConsts<R>& C = *(const MConsts<R>*)a.consts;
    if constexpr (ND == 2 && is_euler_rp<RP>::value) {
      axisym_source_kernel<RP, R><<<launch_grid(a.ntiles_total), kMaxspeedCells, 0, a.stream>>>(
          a.members, a.tiles, a.ntiles_total, C, a.src_phase);
      return cudaGetLastError();
    } else {
      (void)C;
      return cudaErrorNotSupported;
    }
  }
  static cudaError_t maxspeed(const LaunchArgs& a) {
    const MConsts<R>& C = *(const MConsts<R>*)a.consts;
    if constexpr (ND == 3) {
      const long long n = (long long)a.n3[0] * a.n3[1] * a.n3[2];
      maxspeed3_kernel<RP, R><<<(unsigned)((n + 255) / 256), 256, 0, a.stream>>>(a.members, C);
    } else {
      maxspeed_kernel<RP, R, ND><<<launch_grid(a.ntiles_total), kMaxspeedCells, 0, a.stream>>>(
          a.members, a.tiles, a.ntiles_total, C);
    }
    return cudaGetLastError();
  }
};

template <template <typename, int> class RPT, int ND, typename R>
KernelSet make_set(bool has_char) {
  using RP = RPT<R, ND>;
  KernelSet k{};
  k.valid = 1;
  k.M = RP::M;
  k.MW = RP::MW;
  k.MA = RP::MA;
  k.has_char = has_char ? 1 : 0;
  k.classic = &Launchers<RP, R, ND>::classic;
  k.sharp = &Launchers<RP, R, ND>::sharp;
  k.maxspeed = &Launchers<RP, R, ND>::maxspeed;
  k.source = &Launchers<RP, R, ND>::source;
  k.max_bw = classic2d_fits<RP, R>(128) ? 128 : 64;
  constexpr size_t lim = kSmemPerBlock;
  k.sharp_shapes = (sharp_smem_bytes<RP, R, 2, 16, 8, 3>() <= lim ? 1 : 0) |
                   (sharp_smem_bytes<RP, R, 2, 32, 4, 3>() <= lim ? 2 : 0) |
                   (sharp_smem_bytes<RP, R, 2, 32, 8, 3>() <= lim ? 4 : 0) |
                   (sharp_smem_bytes<RP, R, 2, 16, 16, 3>() <= lim ? 8 : 0);
  return k;
}

}  // namespace claw
