// api.cu -- host runtime behind the C ABI of include/clawgpu.h: solver handles,
// batches and the continuous-batching server.  All numerical work happens in
// the fused kernels; this file validates arguments, owns work buffers and
// control blocks, orders work on the caller's stream, captures CUDA graphs of
// step attempts, and runs the step-size autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "claw_common.cuh"
#include "kernels.h"

namespace claw {
// k_common.cu: copy the state of slot ctl->cur into slot dst on the device
cudaError_t launch_select_copy(const Member* mem, const DevCtl* ctl, int dst, size_t bytes,
                               cudaStream_t st);
}  // namespace claw

using namespace claw;

namespace {

thread_local std::string g_err = "no error";

const char* kVersion = "clawgpu 1.0 (sm_103a)";

KernelSet kernels_for(int rp, int nd, int prec) {
  switch (rp) {
    case CLAW_RP_ADVECTION: return claw_kernels_advection(nd, prec);
    case CLAW_RP_ACOUSTICS: return claw_kernels_acoustics(nd, prec);
    case CLAW_RP_SW_ROE: return claw_kernels_sw(nd, prec);
    case CLAW_RP_EULER_ROE: return claw_kernels_euler_roe(nd, prec);
    case CLAW_RP_EULER_HLLE: return claw_kernels_euler_hlle(nd, prec);
    case CLAW_RP_ELASTICITY_FWAVE: return claw_kernels_elasticity(nd, prec);
    case CLAW_RP_EULER_TRACER: return claw_kernels_euler_tracer(nd, prec);
    case CLAW_RP_ACOUSTICS_VC: return claw_kernels_acoustics_vc(nd, prec);
  }
  return KernelSet{};
}

template <typename R>
void fill_consts(const claw_method& m, MConsts<R>& C) {
  std::memset(&C, 0, sizeof(C));
  for (int k = 0; k < 8; ++k) {
    C.p[k] = (R)m.params[k];
    C.inflow[k] = (R)m.inflow[k];
  }
  if (m.rp == CLAW_RP_ACOUSTICS) {
    const double c = std::sqrt(m.params[1] / m.params[0]);
    const double Z = m.params[0] * c;
    C.aco_c = (R)c;
    C.aco_Z = (R)Z;
    C.aco_h = (R)(1.0 / (2.0 * Z));
  }
  C.g = (R)m.params[0];
  C.gamma = (R)m.params[0];
  C.gm1 = (R)(m.params[0] - 1.0);
  C.weno_eps = (R)m.weno_eps;
  C.weno_r = (m.weno_order + 1) / 2;
  C.capa = m.capa_index;
  C.lim = m.lim;
  C.order = m.order;
  C.transverse = m.dim_split ? 0 : m.transverse;
  C.entropy_fix = m.entropy_fix;
  C.char_decomp = m.char_decomp;
  for (int d = 0; d < 3; ++d) {
    C.bc_lo[d] = m.bc_lower[d];
    C.bc_hi[d] = m.bc_upper[d];
  }
}

std::vector<unsigned char> make_consts(const claw_method& m) {
  std::vector<unsigned char> v;
  if (m.prec == CLAW_FP64) {
    v.resize(sizeof(MConsts<double>));
    fill_consts<double>(m, *(MConsts<double>*)v.data());
  } else {
    v.resize(sizeof(MConsts<float>));
    fill_consts<float>(m, *(MConsts<float>*)v.data());
  }
  return v;
}

int num_eqn(int rp, int nd) {
  switch (rp) {
    case CLAW_RP_ADVECTION: return 1;
    case CLAW_RP_ACOUSTICS: return nd + 1;
    case CLAW_RP_SW_ROE: return nd <= 2 ? nd + 1 : 0;
    case CLAW_RP_EULER_ROE:
    case CLAW_RP_EULER_HLLE: return nd <= 2 ? nd + 2 : 0;
    case CLAW_RP_ELASTICITY_FWAVE: return nd <= 2 ? nd + 1 : 0;
    case CLAW_RP_EULER_TRACER: return nd <= 2 ? nd + 3 : 0;
    case CLAW_RP_ACOUSTICS_VC: return nd <= 2 ? nd + 1 : 0;
  }
  return 0;
}

// aux fields the Riemann solver reads
int solver_aux(int rp) {
  return (rp == CLAW_RP_ELASTICITY_FWAVE || rp == CLAW_RP_ACOUSTICS_VC) ? 2 : 0;
}

// validate a method against a dimension; returns an error message or nullptr
const char* check_method(const claw_method& m, int nd) {
  if (nd < 1 || nd > 3) return "ndim must be 1, 2 or 3";
  if (nd == 3 && m.scheme != CLAW_CLASSIC) return "3D grids use the classic scheme";
  if (m.rp < 0 || m.rp > 7) return "unknown Riemann solver";
  if (num_eqn(m.rp, nd) == 0) return "solver not available in this dimension";
  if (m.num_eqn != num_eqn(m.rp, nd)) return "num_eqn does not match the Riemann solver";
  const int na = solver_aux(m.rp);
  if (m.capa_index != -1 && m.capa_index != na)
    return "capa_index must be -1 or the aux field after the solver's own";
  if (m.num_aux != na + (m.capa_index >= 0 ? 1 : 0))
    return "num_aux does not match the Riemann solver (and capacity field)";
  if (m.capa_index >= 0 && nd == 3) return "capacity is for 1D and 2D grids";
  if (m.scheme == CLAW_SHARPCLAW && m.char_decomp && m.rp == CLAW_RP_ACOUSTICS_VC)
    return "no characteristic projection for the varying-medium acoustics solver";
  if (m.scheme != CLAW_CLASSIC && m.scheme != CLAW_SHARPCLAW) return "unknown scheme";
  if (m.prec != CLAW_FP64 && m.prec != CLAW_FP32) return "unknown precision";
  if (m.lim < 0 || m.lim > 4) return "unknown limiter";
  if (m.scheme == CLAW_CLASSIC && m.order != 1 && m.order != 2) return "order must be 1 or 2";
  if (m.transverse < 0 || m.transverse > 2) return "transverse must be 0, 1 or 2";
  if (m.scheme == CLAW_SHARPCLAW &&
      (m.weno_order < 5 || m.weno_order > 17 || m.weno_order % 2 == 0))
    return "weno_order must be odd, 5 to 17";
  if (m.scheme == CLAW_SHARPCLAW && m.time_integrator != CLAW_SSP_RK3 &&
      m.time_integrator != CLAW_SSP104)
    return "unknown time integrator";
  if (m.scheme == CLAW_SHARPCLAW && m.char_decomp && m.rp == CLAW_RP_ELASTICITY_FWAVE)
    return "no characteristic projection for the f-wave elasticity solver";
  if (m.scheme == CLAW_CLASSIC && nd == 2 && m.rp == CLAW_RP_ELASTICITY_FWAVE)
    return "the 2D p-system has normal solves only: use SharpClaw";
  if (m.source != CLAW_SOURCE_NONE && m.source != CLAW_SOURCE_AXISYMMETRIC)
    return "unknown source term";
  if (m.source == CLAW_SOURCE_AXISYMMETRIC &&
      !(nd == 2 && (m.rp == CLAW_RP_EULER_ROE || m.rp == CLAW_RP_EULER_HLLE ||
                    m.rp == CLAW_RP_EULER_TRACER)))
    return "the axisymmetric source needs a 2D Euler system";
  if (m.source_split != CLAW_SPLIT_GODUNOV && m.source_split != CLAW_SPLIT_STRANG)
    return "source_split must be CLAW_SPLIT_GODUNOV or CLAW_SPLIT_STRANG";
  if (m.dim_split != 0 && m.dim_split != 1) return "dim_split must be 0 or 1";
  if (m.dim_split && !(m.scheme == CLAW_CLASSIC && nd == 2))
    return "dimensional splitting is for the classic 2D scheme";
  if (!(m.cfl_desired > 0) || !(m.cfl_max >= m.cfl_desired)) return "need 0 < cfl_desired <= cfl_max";
  if (!(m.dt_max > 0)) return "dt_max must be positive";
  if (m.max_retries < 0) return "max_retries must be >= 0";
  for (int d = 0; d < nd; ++d) {
    if (m.bc_lower[d] < 0 || m.bc_lower[d] > 3 || m.bc_upper[d] < 0 || m.bc_upper[d] > 3)
      return "unknown boundary condition";
    if ((m.bc_lower[d] == CLAW_BC_PERIODIC) != (m.bc_upper[d] == CLAW_BC_PERIODIC))
      return "periodic boundaries must be paired";
  }
  if ((m.rp == CLAW_RP_ACOUSTICS) && !(m.params[0] > 0 && m.params[1] > 0))
    return "acoustics needs rho > 0 and K > 0";
  if ((m.rp == CLAW_RP_SW_ROE) && !(m.params[0] > 0)) return "shallow water needs g > 0";
  if ((m.rp == CLAW_RP_EULER_ROE || m.rp == CLAW_RP_EULER_HLLE) && !(m.params[0] > 1))
    return "Euler needs gamma > 1";
  return nullptr;
}

const char* check_grid(const claw_grid& g, const claw_method& m) {
  if (g.ndim < 1 || g.ndim > 3) return "ndim must be 1, 2 or 3";
  // the ghost layer (WENO half-width for SharpClaw) must fit in the grid
  const int need = m.scheme == CLAW_SHARPCLAW ? std::max(4, (m.weno_order + 1) / 2) : 4;
  for (int d = 0; d < g.ndim; ++d) {
    if (g.n[d] < need) return "too few cells in a direction for the ghost layer";
    if (g.n[d] > (int64_t)INT_MAX / 2) return "too many cells in one direction";
    if (!(g.upper[d] > g.lower[d])) return "upper must exceed lower";
  }
  if (m.source == CLAW_SOURCE_AXISYMMETRIC && !(g.ndim == 2 && g.lower[1] >= 0.0))
    return "the axisymmetric source needs r = y >= 0 on the grid";
  return nullptr;
}

// ma: the solver's aux fields (the 1D classic tile depends on them)
int tiles_of(int scheme, int nd, int prec, int ma, int nx, int ny, int bw, int h) {
  if (scheme == CLAW_CLASSIC)
    return nd == 1 ? classic1d_tiles(nx, prec, ma) : classic2d_tiles(nx, ny, bw, h);
  if (nd == 1) return sharp_tiles(nx, 1, kSharpTX1, 1);
  int tx, ty;
  sharp2d_shape(bw, h, tx, ty);
  return sharp_tiles(nx, ny, tx, ty);
}

// The launch shape a scheme starts with: the 2D SharpClaw default tile, or
// the classic defaults (bw, h) the caller holds.
void default_shape(const claw_method& m, int nd, int& bw, int& h) {
  if (m.scheme != CLAW_SHARPCLAW) return;
  bw = nd == 1 ? kSharpTX1 : kSharpTX2;
  h = nd == 1 ? 1 : kSharpTY2;
}

// Candidate launch shapes of the fused step: classic 2D tile shapes (bw, h)
// for strips of 60 and 124 columns and a range of chunk heights; classic 1D
// work modes (h = kWork1dTiles / kWork1dUnits); the 2D SharpClaw tiles of
// the fifth-order stage (kSharpShapes2).  Every candidate gives the same
// bits; they differ only in speed.
std::vector<std::pair<int, int>> tile_candidates(const KernelSet& ks, const claw_method& m,
                                                 int nd) {
  std::vector<std::pair<int, int>> c;
  const int max_bw = ks.max_bw;
  if (m.scheme == CLAW_SHARPCLAW) {
    if (nd == 2 && m.weno_order == 5) {
      for (int i = 0; i < 4; ++i)
        if (i == 0 || ((ks.sharp_shapes >> i) & 1))
          c.push_back({kSharpShapes2[i][0], kSharpShapes2[i][1]});
    } else
      c.push_back(nd == 1 ? std::make_pair(kSharpTX1, 1) : std::make_pair(kSharpTX2, kSharpTY2));
    return c;
  }
  if (nd == 1) {
    c.push_back({0, kWork1dTiles});
    c.push_back({0, kWork1dUnits});
    return c;
  }
  for (int bw : {64, 128}) {
    if (bw > max_bw) continue;
    for (int h : {8, 12, 16, 21, 24, 32, 41, 48, 64, 96, 128}) c.push_back({bw, h});
  }
  return c;
}

// Why a launch shape set by hand cannot be taken (null when it can).
const char* bad_shape(const KernelSet& ks, const claw_method& m, int nd, int bw, int h) {
  const int max_bw = ks.max_bw;
  if (m.scheme == CLAW_SHARPCLAW) {
    for (const auto& pr : tile_candidates(ks, m, nd))
      if (pr.first == bw && pr.second == h) return nullptr;
    return nd == 2 ? "bad SharpClaw tile (WENO5: 16x8, 32x4, 32x8, 16x16; higher orders: 16x8)"
                   : "the 1D SharpClaw tile is 128 x 1";
  }
  if (nd == 1)
    return h == kWork1dTiles || h == kWork1dUnits
               ? nullptr
               : "bad 1D work mode (1 whole tiles, 2 single units)";
  if ((bw != 64 && bw != 128) || bw > max_bw || h < 1) return "bad tile shape";
  return nullptr;
}

// One trial attempt of a tuning candidate: the classic step, or the first
// stage of the SharpClaw integrator (it writes only a work buffer)
cudaError_t trial_launch(const KernelSet& ks, const claw_method& m, LaunchArgs a) {
  if (m.scheme == CLAW_CLASSIC) return ks.classic(a);
  const StageOp* ops;
  stage_table(m.time_integrator, &ops);
  a.stage = 0;
  a.stage_op = ops;
  return ks.sharp(a);
}

// Time the candidate shapes on a table of members (hm: host copies whose
// control blocks are the real ones) and return the fastest in bw, h.  The trial attempts run on dry copies of the control
// blocks, so every t, dt and buffer rotation stays as it was (a trial writes
// only each member's next work buffer, which the next real attempt
// rewrites); only the classic step runs, no source step.
cudaError_t tune_members(const KernelSet& ks, int nd, const claw_method& m,
                         const std::vector<Member>& hm, const void* consts, cudaStream_t st,
                         int& bw, int& h) {
  const int n = (int)hm.size();
  if (n == 0) return cudaSuccess;
  DevCtl* dctl = nullptr;
  Member* dmem = nullptr;
  Tile* dtiles = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&dctl, sizeof(DevCtl) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dmem, sizeof(Member) * n);
  // copies of the real control blocks (gathered through the real table)
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dmem, hm.data(), sizeof(Member) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_gather_ctl(dmem, n, dctl, st);
  if (e == cudaSuccess) e = launch_set_dry_n(dctl, n, 1, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  std::vector<Member> tm(hm);
  for (int k = 0; k < n; ++k) {
    tm[k].ctl = dctl + k;
    tm[k].qpre = nullptr;  // trial attempts read Q^n itself
  }
  size_t cap = 0;
  float best = 1e30f;
  int bb = bw, bh = h;
  for (const auto& pr : tile_candidates(ks, m, nd)) {
    if (e != cudaSuccess) break;
    std::vector<Tile> tt;
    for (int k = 0; k < n; ++k) {
      tm[k].ntiles = tiles_of(m.scheme, nd, m.prec, ks.MA, tm[k].nx, tm[k].ny, pr.first,
                              pr.second);
      for (int t = 0; t < tm[k].ntiles; ++t) tt.push_back(Tile{k, t});
    }
    if (tt.size() > cap) {
      if (dtiles) cudaFree(dtiles);
      cap = tt.size();
      if ((e = cudaMalloc(&dtiles, sizeof(Tile) * cap)) != cudaSuccess) break;
    }
    if ((e = cudaMemcpyAsync(dmem, tm.data(), sizeof(Member) * n, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      break;
    if ((e = cudaMemcpyAsync(dtiles, tt.data(), sizeof(Tile) * tt.size(), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess)
      break;
    LaunchArgs a{dmem, dtiles, (int)tt.size(), consts, pr.first, pr.second, 0, st};
    a.nmembers = n;
    if ((e = trial_launch(ks, m, a)) != cudaSuccess) {  // warm-up
      // a shape this solver does not have, or that the device cannot launch
      // (configuration errors leave the context usable): skip it
      if (e != cudaErrorNotSupported && e != cudaErrorInvalidValue &&
          e != cudaErrorLaunchOutOfResources && e != cudaErrorInvalidConfiguration)
        break;
      e = cudaSuccess;
      continue;
    }
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) trial_launch(ks, m, a);
    cudaEventRecord(e1, st);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;  // tt, tm stay alive till here
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bb = pr.first;
      bh = pr.second;
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (dtiles) cudaFree(dtiles);
  if (dmem) cudaFree(dmem);
  if (dctl) cudaFree(dctl);
  if (e != cudaSuccess) return e;
  if (nd == 2) bw = bb;
  h = bh;
  return cudaSuccess;
}

int maxspeed_tiles(int nx, int ny) {
  const long long n = (long long)nx * ny;
  return (int)((n + kMaxspeedCells - 1) / kMaxspeedCells);
}

// state buffers a scheme rotates through: classic Q^n, Q^{n+1}; SSP-RK3 adds
// one stage state; SSP(10,4) two (its two low-storage registers)
int nbuf_of(const claw_method& m) {
  if (m.scheme == CLAW_CLASSIC) return m.dim_split ? 3 : 2;
  return m.time_integrator == CLAW_SSP104 ? 4 : 3;
}
// a Strang-split source needs one more state: Q^n after the first half step
int pre_buffers(const claw_method& m) {
  return (m.source != CLAW_SOURCE_NONE && m.source_split == CLAW_SPLIT_STRANG) ? 1 : 0;
}

DevCtl make_ctl(const claw_method& m, const claw_grid& g, int nbuf, double t0, double t_end) {
  DevCtl c;
  std::memset(&c, 0, sizeof(c));
  c.t = t0;
  c.t_end = t_end;
  c.dt_max = m.dt_max;
  c.cfl_desired = m.cfl_desired;
  c.cfl_max = m.cfl_max;
  c.dx[0] = (g.upper[0] - g.lower[0]) / (double)g.n[0];
  c.dx[1] = g.ndim >= 2 ? (g.upper[1] - g.lower[1]) / (double)g.n[1] : 1.0;
  c.dx[2] = g.ndim == 3 ? (g.upper[2] - g.lower[2]) / (double)g.n[2] : 1.0;
  for (int d = 0; d < 3; ++d) c.idx[d] = 1.0 / c.dx[d];
  c.dt_init = m.dt_initial;
  c.max_steps = LLONG_MAX;
  c.nbuf = nbuf;
  c.accept_shift = ((m.scheme == CLAW_SHARPCLAW && m.time_integrator == CLAW_SSP104) ||
                    (m.scheme == CLAW_CLASSIC && m.dim_split))
                       ? 2
                       : 1;
  for (int d = 0; d < 3; ++d) c.lo[d] = d < g.ndim ? g.lower[d] : 0.0;
  c.max_retries = m.max_retries;
  c.ndim = g.ndim;
  c.done = (t0 >= t_end) ? 1 : 0;
  return c;
}

size_t cells_of(const claw_grid& g) {
  return (size_t)g.n[0] * (g.ndim >= 2 ? (size_t)g.n[1] : 1) * (g.ndim == 3 ? (size_t)g.n[2] : 1);
}
size_t state_bytes_of(const claw_method& m, const claw_grid& g) {
  const size_t es = m.prec == CLAW_FP64 ? 8 : 4;
  return cells_of(g) * m.num_eqn * es;
}
size_t aux_bytes_of(const claw_method& m, const claw_grid& g) {
  const size_t es = m.prec == CLAW_FP64 ? 8 : 4;
  return cells_of(g) * m.num_aux * es;
}
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

void fill_info(const DevCtl& c, claw_step_info* info) {
  if (!info) return;
  info->t = c.t;
  info->dt_used = c.dt_used;
  info->dt_next = c.dt;
  info->cfl = c.nu_last;
  info->cfl_max_seen = c.nu_max_seen;
  info->steps = c.steps;
  info->rejects = c.rejects;
  info->accepted = c.accepted;
  info->status = c.status;
}

// Launch one attempt: classic, one kernel (two sweeps when dimensionally
// split); SharpClaw, one kernel per stage; with a source, its fractional
// steps over the cell tiles (mtiles): Godunov, after the step; Strang, half
// before the step (into Member::qpre) and half after it.
cudaError_t launch_attempt(const KernelSet& ks, const claw_method& m, const Member* mem,
                           const Tile* tiles, int ntiles, const void* consts, int bw, int h,
                           cudaStream_t st, const Tile* mtiles = nullptr, int nmtiles = 0,
                           int nmembers = 1, const int* n3 = nullptr, void* work3 = nullptr,
                           size_t work3_bytes = 0) {
  LaunchArgs a{mem, tiles, ntiles, consts, bw, h, 0, st};
  a.nmembers = nmembers;
  if (n3) {
    a.n3[0] = n3[0];
    a.n3[1] = n3[1];
    a.n3[2] = n3[2];
  }
  a.work3 = work3;
  a.work3_bytes = work3_bytes;
  cudaError_t e = cudaSuccess;
  const bool strang = m.source != CLAW_SOURCE_NONE && m.source_split == CLAW_SPLIT_STRANG;
  LaunchArgs b{mem, mtiles, nmtiles, consts, 0, 0, 0, st};
  if (strang) {
    b.src_phase = 1;  // S(dt/2) Q^n into the pre-source buffer the step reads
    if ((e = ks.source(b)) != cudaSuccess) return e;
  }
  if (m.scheme == CLAW_CLASSIC) {
    if (m.dim_split) {
      a.sweep = 1;
      if ((e = ks.classic(a)) != cudaSuccess) return e;
      a.sweep = 2;
    }
    e = ks.classic(a);
  } else {
    const StageOp* ops;
    const int ns = stage_table(m.time_integrator, &ops);
    for (int s = 0; s < ns && e == cudaSuccess; ++s) {
      a.stage = s;
      a.stage_op = ops + s;
      e = ks.sharp(a);
    }
  }
  if (e != cudaSuccess || m.source == CLAW_SOURCE_NONE) return e;
  b.src_phase = strang ? 2 : 0;
  if ((e = ks.source(b)) != cudaSuccess) return e;
  return launch_source_mark(mem, nmembers, st);
}

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

void claw::set_last_error(const char* msg) { g_err = msg; }

// the same validation, constants and kernel sets for the library's other
// translation units (the allocation-free step)
const char* claw::validate_method(const claw_method& m, int nd) { return check_method(m, nd); }
const char* claw::validate_grid(const claw_grid& g, const claw_method& m) {
  return check_grid(g, m);
}
std::vector<unsigned char> claw::method_consts(const claw_method& m) { return make_consts(m); }
claw::KernelSet claw::kernels_of(int rp, int nd, int prec) { return kernels_for(rp, nd, prec); }

// ===========================================================================
// single-grid solver
// ===========================================================================
struct claw_solver {
  claw_method m;
  claw_grid g;
  int nd = 1, prec = 0, nbuf = 2;
  int faces = 0;  // classic step on the per-face path (capacity / media-aware transverse)
  KernelSet ks{};
  std::vector<unsigned char> consts;
  cudaStream_t ustream = nullptr, st = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  void* q_user = nullptr;
  const void* aux = nullptr;
  void* work = nullptr;
  size_t sbytes = 0;
  DevCtl* d_ctl = nullptr;
  DevCtl* h_ctl = nullptr;  // pinned
  Member* d_mem = nullptr;
  Member h_mem{};
  DevCtl* d_ctl_tune = nullptr;
  Member* d_mem_tune = nullptr;
  double* d_part = nullptr;
  double* h_part = nullptr;  // pinned
  int npart = 0;
  int ntiles = 0, bw = 128, h = 32;
  int tuned = 0;
  void* work3 = nullptr;  // 3D per-face arrays
  size_t work3_bytes = 0;
  cudaGraphExec_t gexec = nullptr;
  int gk = 0;
  int bound = 0;
  std::string err;
};

namespace {

claw_status fail(claw_solver* s, const char* what, cudaError_t e = cudaSuccess) {
  std::string msg = what;
  if (e != cudaSuccess) {
    msg += ": ";
    msg += cudaGetErrorString(e);
  }
  if (s) s->err = msg;
  g_err = msg;
  return e != cudaSuccess ? CLAW_ECUDA : CLAW_EINVAL;
}

#define SCK(call)                                      \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return fail(s, #call, e_);  \
  } while (0)

cudaError_t enter(claw_solver* s) {
  if (s->st == s->ustream) return cudaSuccess;
  cudaError_t e = cudaEventRecord(s->ev_a, s->ustream);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(s->st, s->ev_a, 0);
}
cudaError_t leave(claw_solver* s) {
  if (s->st == s->ustream) return cudaSuccess;
  cudaError_t e = cudaEventRecord(s->ev_b, s->st);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(s->ustream, s->ev_b, 0);
}

cudaError_t solver_attempt(claw_solver* s, cudaStream_t st) {
  if (s->nd == 3) {
    LaunchArgs a{s->d_mem, nullptr, s->ntiles, s->consts.data(), 0, 0, 0, st,
                 {(int)s->g.n[0], (int)s->g.n[1], (int)s->g.n[2]}, s->work3, s->work3_bytes};
    return s->ks.classic(a);
  }
  const int n3[3] = {(int)s->g.n[0], (int)s->g.n[1], (int)s->g.n[2]};
  return launch_attempt(s->ks, s->m, s->d_mem, nullptr, s->ntiles, s->consts.data(), s->bw,
                        s->h, st, nullptr, maxspeed_tiles(s->h_mem.nx, s->h_mem.ny), 1, n3,
                        s->work3, s->work3_bytes);
}

cudaError_t read_ctl(claw_solver* s) {
  cudaError_t e = cudaMemcpyAsync(s->h_ctl, s->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s->st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s->st);
}

cudaError_t upload_member(claw_solver* s) {
  s->h_mem.ntiles = s->ntiles;
  return cudaMemcpyAsync(s->d_mem, &s->h_mem, sizeof(Member), cudaMemcpyHostToDevice, s->st);
}

void drop_graph(claw_solver* s) {
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  s->gexec = nullptr;
  s->gk = 0;
}

cudaError_t build_graph(claw_solver* s, int k) {
  drop_graph(s);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < k && e == cudaSuccess; ++i) e = solver_attempt(s, s->st);
  cudaError_t e2 = cudaStreamEndCapture(s->st, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return e;
  }
  if (e2 != cudaSuccess) return e2;
  e = cudaGraphInstantiate(&s->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e == cudaSuccess) s->gk = k;
  return e;
}

// Time candidate (bw, h) shapes of the 2D classic kernel on the bound state
// with a dry control block (attempts leave t, dt and the state untouched) and
// keep the fastest.
cudaError_t autotune(claw_solver* s) {
  if (s->m.scheme == CLAW_CLASSIC && s->nd == 1 && !s->faces) {
    // 1D: how warps take work (whole tiles or single units)
    int bw = s->bw, h = s->h;
    cudaError_t e = tune_members(s->ks, 1, s->m, {s->h_mem}, s->consts.data(), s->st, bw, h);
    if (e != cudaSuccess) return e;
    s->h = h;
    s->tuned = 1;
    drop_graph(s);
    return cudaSuccess;
  }
  if (s->m.scheme == CLAW_SHARPCLAW && s->nd == 2 && s->m.weno_order == 5) {
    // the SharpClaw tile, timed on the first stage with a dry control block
    int bw = s->bw, h = s->h;
    cudaError_t e = tune_members(s->ks, 2, s->m, {s->h_mem}, s->consts.data(), s->st, bw, h);
    if (e != cudaSuccess) return e;
    s->bw = bw;
    s->h = h;
    s->ntiles = tiles_of(s->m.scheme, 2, s->prec, s->ks.MA, (int)s->g.n[0], (int)s->g.n[1],
                         bw, h);
    s->tuned = 1;
    drop_graph(s);
    return upload_member(s);
  }
  if (s->m.scheme != CLAW_CLASSIC || s->nd != 2 || s->faces) {
    s->tuned = 1;
    return cudaSuccess;
  }
  cudaError_t e = cudaSuccess;
  if (!s->d_ctl_tune) {
    if ((e = cudaMalloc(&s->d_ctl_tune, sizeof(DevCtl))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&s->d_mem_tune, sizeof(Member))) != cudaSuccess) return e;
  }
  if ((e = cudaMemcpyAsync(s->d_ctl_tune, s->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToDevice,
                           s->st)) != cudaSuccess)
    return e;
  if ((e = launch_set_dry(s->d_ctl_tune, 1, s->st)) != cudaSuccess) return e;
  if ((e = launch_set_t_end(s->d_ctl_tune, 1, INFINITY, 0, s->st)) != cudaSuccess) return e;
  Member mt = s->h_mem;
  mt.ctl = s->d_ctl_tune;
  mt.qpre = nullptr;  // trial launches read Q^n itself
  const int nx = (int)s->g.n[0], ny = (int)s->g.n[1];
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int bws[2] = {64, 128};
  // fixed heights, plus for each k the lowest height whose tile count fits in
  // k x (number of SMs), k = 1..8: whole waves at any residency
  std::vector<std::pair<int, int>> cand;
  for (int bw : bws) {
    if (bw > s->ks.max_bw) continue;
    for (int h : {8, 16, 32, 64, 128})
      if (h <= 2 * ny) cand.push_back({bw, h});
    for (int k = 1; k <= 8; ++k) {
      if (nsm <= 0) break;
      int h = 4;
      while (h < ny && classic2d_tiles(nx, ny, bw, h) > k * nsm) ++h;
      bool seen = false;
      for (auto& pr : cand) seen |= (pr.first == bw && pr.second == h);
      if (!seen) cand.push_back({bw, h});
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bb = s->ks.max_bw, bh = 32;
  for (const auto& pr : cand) {
    const int bw = pr.first, h = pr.second;
    const int nt = classic2d_tiles(nx, ny, bw, h);
    mt.ntiles = nt;
    if ((e = cudaMemcpyAsync(s->d_mem_tune, &mt, sizeof(Member), cudaMemcpyHostToDevice,
                             s->st)) != cudaSuccess)
      break;
    LaunchArgs a{s->d_mem_tune, nullptr, nt, s->consts.data(), bw, h, 0, s->st};
    if ((e = s->ks.classic(a)) != cudaSuccess) break;  // warm-up
    cudaEventRecord(e0, s->st);
    for (int r = 0; r < 3; ++r) s->ks.classic(a);
    cudaEventRecord(e1, s->st);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bb = bw;
      bh = h;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  s->bw = bb;
  s->h = bh;
  s->ntiles = classic2d_tiles(nx, ny, bb, bh);
  s->tuned = 1;
  drop_graph(s);
  return upload_member(s);
}

void free_bound(claw_solver* s) {
  drop_graph(s);
  if (s->work) cudaFree(s->work);
  if (s->work3) cudaFree(s->work3);
  s->work3 = nullptr;
  if (s->d_ctl) cudaFree(s->d_ctl);
  if (s->d_mem) cudaFree(s->d_mem);
  if (s->d_ctl_tune) cudaFree(s->d_ctl_tune);
  if (s->d_mem_tune) cudaFree(s->d_mem_tune);
  if (s->d_part) cudaFree(s->d_part);
  if (s->h_ctl) cudaFreeHost(s->h_ctl);
  if (s->h_part) cudaFreeHost(s->h_part);
  s->work = nullptr;
  s->d_ctl = nullptr;
  s->d_mem = nullptr;
  s->d_ctl_tune = nullptr;
  s->d_mem_tune = nullptr;
  s->d_part = nullptr;
  s->h_ctl = nullptr;
  s->h_part = nullptr;
  s->bound = 0;
}

claw_status sync_state_impl(claw_solver* s) {
  SCK(read_ctl(s));
  if (s->h_ctl->cur != 0) {
    const unsigned char* src = (const unsigned char*)s->h_mem.q[s->h_ctl->cur];
    SCK(cudaMemcpyAsync(s->q_user, src, s->sbytes, cudaMemcpyDeviceToDevice, s->st));
    SCK(launch_reset_cur(s->d_ctl, s->st));
    SCK(read_ctl(s));
  }
  return CLAW_OK;
}

}  // namespace

extern "C" {

claw_status claw_method_init(claw_method* m, int rp, int ndim) {
  if (!m) return CLAW_EINVAL;
  std::memset(m, 0, sizeof(*m));
  if (ndim < 1 || ndim > 3) {
    g_err = "ndim must be 1, 2 or 3";
    return CLAW_EINVAL;
  }
  if (rp < 0 || rp > 7 || num_eqn(rp, ndim) == 0) {
    g_err = "unknown Riemann solver for this dimension";
    return CLAW_EINVAL;
  }
  // the 2D p-system has normal solves only (Sec. 7.3 uses SharpClaw)
  m->scheme = (rp == CLAW_RP_ELASTICITY_FWAVE && ndim == 2) ? CLAW_SHARPCLAW : CLAW_CLASSIC;
  m->rp = rp;
  m->lim = CLAW_LIM_MC;
  m->prec = CLAW_FP64;
  m->order = 2;
  m->transverse = ndim >= 2 ? 2 : 0;
  m->weno_order = 5;
  m->char_decomp = (rp == CLAW_RP_ELASTICITY_FWAVE || rp == CLAW_RP_ACOUSTICS_VC) ? 0 : 1;
  m->entropy_fix = 1;
  m->max_retries = 8;
  m->cfl_desired = 0.9;
  m->cfl_max = 1.0;
  m->dt_initial = 0.0;
  m->dt_max = 1e30;
  m->weno_eps = 1e-6;
  for (int d = 0; d < 3; ++d) m->bc_lower[d] = m->bc_upper[d] = CLAW_BC_PERIODIC;
  switch (rp) {
    case CLAW_RP_ADVECTION: m->params[0] = 1.0; m->params[1] = 1.0; break;
    case CLAW_RP_ACOUSTICS: m->params[0] = 1.0; m->params[1] = 1.0; break;
    case CLAW_RP_SW_ROE: m->params[0] = 1.0; break;
    case CLAW_RP_EULER_ROE:
    case CLAW_RP_EULER_HLLE: m->params[0] = 1.4; break;
    default: break;
  }
  m->num_eqn = num_eqn(rp, ndim);
  m->num_aux = solver_aux(rp);
  m->capa_index = -1;
  m->source_split = CLAW_SPLIT_GODUNOV;
  return CLAW_OK;
}

claw_status claw_solver_create(const claw_method* m, const claw_grid* g, void* stream,
                               claw_solver** out) {
  if (!m || !g || !out) return fail(nullptr, "null argument");
  *out = nullptr;
  if (const char* why = check_grid(*g, *m)) return fail(nullptr, why);
  if (const char* why = check_method(*m, g->ndim)) return fail(nullptr, why);
  KernelSet ks = kernels_for(m->rp, g->ndim, m->prec);
  if (!ks.valid) return fail(nullptr, "no kernels for this solver/dimension/precision");
  claw_solver* s = new claw_solver();
  s->m = *m;
  s->g = *g;
  if (g->ndim == 1) s->g.n[1] = 1;
  if (g->ndim <= 2) s->g.n[2] = 1;
  s->nd = g->ndim;
  s->prec = m->prec;
  s->nbuf = nbuf_of(*m);
  s->ks = ks;
  s->bw = std::min(s->bw, ks.max_bw);
  default_shape(*m, s->nd, s->bw, s->h);
  s->consts = make_consts(*m);
  s->ustream = (cudaStream_t)stream;
  s->sbytes = state_bytes_of(*m, s->g);
  // work goes straight onto a caller's stream; the legacy default stream
  // cannot be captured into a graph, so NULL gets a private stream ordered
  // against it by events
  cudaError_t e = cudaSuccess;
  if (s->ustream) s->st = s->ustream;
  else e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_a, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_b, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    claw_status st = fail(s, "stream/event creation", e);
    claw_solver_destroy(s);
    return st;
  }
  s->faces = (m->scheme == CLAW_CLASSIC && s->nd <= 2 &&
              (m->capa_index >= 0 || (s->nd == 2 && m->rp == CLAW_RP_ACOUSTICS_VC)))
                 ? 1
                 : 0;
  if (s->faces) s->tuned = 1;  // no tile shapes to choose
  s->ntiles = s->nd == 3 ? classic3d_update_blocks(cells_of(s->g))
             : s->faces    ? (int)((cells_of(s->g) + 255) / 256)
                           : tiles_of(m->scheme, s->nd, s->prec, s->ks.MA, (int)s->g.n[0],
                             (int)s->g.n[1], s->bw, s->h);
  *out = s;
  return CLAW_OK;
}

claw_status claw_bind_state(claw_solver* s, void* q_dev, const void* aux_dev, double t0) {
  if (!s) return fail(nullptr, "null solver");
  if (!q_dev) return fail(s, "q_dev is NULL");
  if (s->m.num_aux > 0 && !aux_dev) return fail(s, "this solver needs aux fields");
  free_bound(s);
  s->q_user = q_dev;
  s->aux = aux_dev;
  const int npre = pre_buffers(s->m);
  SCK(cudaMalloc(&s->work, s->sbytes * (s->nbuf - 1 + npre)));
  if (s->faces) {
    s->work3_bytes = faces_work_bytes(s->nd, (int)s->g.n[0], (int)s->g.n[1], s->m.num_eqn,
                                      s->prec);
    SCK(cudaMalloc(&s->work3, s->work3_bytes));
  }
  if (s->nd == 3) {
    s->work3_bytes = classic3d_work_bytes((int)s->g.n[0], (int)s->g.n[1], (int)s->g.n[2],
                                          s->m.num_eqn, s->prec);
    SCK(cudaMalloc(&s->work3, s->work3_bytes));
  }
  SCK(cudaMalloc(&s->d_ctl, sizeof(DevCtl)));
  SCK(cudaMalloc(&s->d_mem, sizeof(Member)));
  SCK(cudaMallocHost(&s->h_ctl, sizeof(DevCtl)));
  const long long ncell = (long long)cells_of(s->g);
  s->npart = (int)std::min<long long>(1024, (ncell + kTotalsThreads - 1) / kTotalsThreads);
  SCK(cudaMalloc(&s->d_part, sizeof(double) * 2 * s->npart * s->m.num_eqn));
  SCK(cudaMallocHost(&s->h_part, sizeof(double) * 2 * s->npart * s->m.num_eqn));
  std::memset(&s->h_mem, 0, sizeof(Member));
  s->h_mem.q[0] = q_dev;
  s->h_mem.q[1] = s->work;
  for (int j = 2; j < s->nbuf; ++j)
    s->h_mem.q[j] = (void*)((unsigned char*)s->work + (size_t)(j - 1) * s->sbytes);
  if (npre) s->h_mem.qpre = (void*)((unsigned char*)s->work + (size_t)(s->nbuf - 1) * s->sbytes);
  s->h_mem.aux = aux_dev;
  s->h_mem.nx = (int)s->g.n[0];
  s->h_mem.ny = (int)s->g.n[1];
  s->h_mem.nz = (int)s->g.n[2];
  s->h_mem.work3 = s->work3;
  s->h_mem.ctl = s->d_ctl;
  DevCtl c = make_ctl(s->m, s->g, s->nbuf, t0, INFINITY);
  SCK(enter(s));
  SCK(cudaMemcpyAsync(s->d_ctl, &c, sizeof(DevCtl), cudaMemcpyHostToDevice, s->st));
  SCK(upload_member(s));
  // first dt from the wave speeds of Q^0 (or dt_initial)
  LaunchArgs a{s->d_mem, nullptr, maxspeed_tiles(s->h_mem.nx, s->h_mem.ny), s->consts.data(), 0,
               0, 0, s->st, {(int)s->g.n[0], (int)s->g.n[1], (int)s->g.n[2]}, nullptr, 0};
  SCK(s->ks.maxspeed(a));
  SCK(launch_dt_init(s->d_ctl, 1, s->st));
  SCK(leave(s));
  SCK(cudaStreamSynchronize(s->st));
  s->bound = 1;
  return CLAW_OK;
}

claw_status claw_solver_tune(claw_solver* s, int mode, int* bw, int* h) {
  if (!s || !s->bound) return fail(s, "solver not bound");
  if (mode == 0) {
    SCK(enter(s));
    SCK(autotune(s));
    SCK(leave(s));
  } else {
    if (s->m.scheme == CLAW_CLASSIC && s->nd == 1 && h &&
        (*h == kWork1dTiles || *h == kWork1dUnits)) {
      s->h = *h;
      s->tuned = 1;
      drop_graph(s);
      if (bw) *bw = s->bw;
      SCK(cudaStreamSynchronize(s->st));
      return CLAW_OK;
    }
    if (!bw || !h) return fail(s, "bad tile shape");
    if (const char* why = bad_shape(s->ks, s->m, s->nd, *bw, *h)) return fail(s, why);
    s->bw = *bw;
    s->h = *h;
    if (s->nd != 3 && !s->faces)
      s->ntiles = tiles_of(s->m.scheme, s->nd, s->prec, s->ks.MA, (int)s->g.n[0],
                           (int)s->g.n[1], s->bw, s->h);
    s->tuned = 1;
    drop_graph(s);
    SCK(enter(s));
    SCK(upload_member(s));
    SCK(leave(s));
  }
  if (bw) *bw = s->bw;
  if (h) *h = s->h;
  SCK(cudaStreamSynchronize(s->st));
  return CLAW_OK;
}

claw_status claw_set_t_end(claw_solver* s, double t_end, int64_t max_steps) {
  if (!s || !s->bound) return fail(s, "solver not bound");
  SCK(enter(s));
  SCK(launch_set_t_end(s->d_ctl, 1, t_end, (long long)max_steps, s->st));
  SCK(leave(s));
  return CLAW_OK;
}

claw_status claw_advance(claw_solver* s, int n) {
  if (!s || !s->bound) return fail(s, "solver not bound");
  if (n < 0) return fail(s, "n must be >= 0");
  SCK(enter(s));
  for (int i = 0; i < n; ++i) SCK(solver_attempt(s, s->st));
  SCK(leave(s));
  return CLAW_OK;
}

claw_status claw_step(claw_solver* s, double dt, claw_step_info* info) {
  if (!s || !s->bound) return fail(s, "solver not bound");
  SCK(enter(s));
  SCK(launch_set_t_end(s->d_ctl, 1, INFINITY, 0, s->st));
  if (dt > 0) {
    SCK(launch_force_dt(s->d_ctl, dt, s->st));
    SCK(solver_attempt(s, s->st));
    SCK(read_ctl(s));
  } else {
    for (int tries = 0; tries <= s->m.max_retries; ++tries) {
      SCK(solver_attempt(s, s->st));
      SCK(read_ctl(s));
      if (s->h_ctl->accepted || s->h_ctl->done) break;
    }
  }
  SCK(leave(s));
  fill_info(*s->h_ctl, info);
  return s->h_ctl->status;
}

claw_status claw_evolve_to_time(claw_solver* s, double t_end, int64_t max_steps, int use_graph,
                                claw_step_info* info) {
  if (!s || !s->bound) return fail(s, "solver not bound");
  SCK(enter(s));
  if (!s->tuned) SCK(autotune(s));
  SCK(launch_set_t_end(s->d_ctl, 1, t_end, (long long)max_steps, s->st));
  const int GK = 16;
  if (use_graph && s->gk != GK) SCK(build_graph(s, GK));
  long long launched = 0;
  for (;;) {
    SCK(read_ctl(s));
    const DevCtl& c = *s->h_ctl;
    if (c.done) break;
    // attempts left: the steps to t_end at the current dt (at least one)
    double left = (c.dt > 0) ? (c.t_end - c.t) / c.dt : 1.0;
    long long k = (long long)std::ceil(std::min(left, 1e9)) + 1;
    if (max_steps > 0) k = std::min<long long>(k, c.max_steps - c.steps);
    k = std::max<long long>(1, std::min<long long>(k, 256));
    if (use_graph) {
      const long long reps = (k + GK - 1) / GK;
      for (long long r = 0; r < reps; ++r) SCK(cudaGraphLaunch(s->gexec, s->st));
      launched += reps * GK;
    } else {
      for (long long i = 0; i < k; ++i) SCK(solver_attempt(s, s->st));
      launched += k;
    }
    if (launched > (1LL << 40)) return fail(s, "evolve made no progress");
  }
  claw_status st = sync_state_impl(s);
  if (st != CLAW_OK) return st;
  SCK(leave(s));
  fill_info(*s->h_ctl, info);
  return s->h_ctl->status;
}

claw_status claw_get_info(claw_solver* s, claw_step_info* info) {
  if (!s || !s->bound) return fail(s, "solver not bound");
  SCK(enter(s));
  SCK(read_ctl(s));
  SCK(leave(s));
  fill_info(*s->h_ctl, info);
  return CLAW_OK;
}

claw_status claw_current_state(claw_solver* s, void** q_cur) {
  if (!s || !s->bound || !q_cur) return fail(s, "solver not bound");
  SCK(enter(s));
  SCK(read_ctl(s));
  SCK(leave(s));
  *q_cur = s->h_mem.q[s->h_ctl->cur];
  return CLAW_OK;
}

claw_status claw_sync_state(claw_solver* s) {
  if (!s || !s->bound) return fail(s, "solver not bound");
  SCK(enter(s));
  claw_status st = sync_state_impl(s);
  if (st != CLAW_OK) return st;
  SCK(leave(s));
  return CLAW_OK;
}

claw_status claw_conserved_totals(claw_solver* s, double* out) {
  if (!s || !s->bound || !out) return fail(s, "solver not bound");
  SCK(enter(s));
  SCK(read_ctl(s));
  const void* q = s->h_mem.q[s->h_ctl->cur];
  const long long ncell = (long long)cells_of(s->g);
  const int M = s->m.num_eqn;
  // capacity-form differencing conserves sum_i kappa_i Q_i
  const void* kappa =
      s->m.capa_index >= 0
          ? (const void*)((const unsigned char*)s->aux +
                          (size_t)s->m.capa_index * ncell * (s->prec == CLAW_FP64 ? 8 : 4))
          : nullptr;
  SCK(launch_totals(q, kappa, s->prec, ncell, M, s->d_part, s->npart, s->st));
  SCK(cudaMemcpyAsync(s->h_part, s->d_part, sizeof(double) * 2 * s->npart * M,
                      cudaMemcpyDeviceToHost, s->st));
  SCK(cudaStreamSynchronize(s->st));
  SCK(leave(s));
  double dV = s->h_ctl->dx[0];
  for (int d = 1; d < s->nd; ++d) dV *= s->h_ctl->dx[d];
  for (int k = 0; k < M; ++k) {
    double sum = 0.0, comp = 0.0;
    for (int b = 0; b < s->npart; ++b) {
      const double* pr = s->h_part + ((size_t)k * s->npart + b) * 2;
      for (int j = 0; j < 2; ++j) {
        const double x = pr[j];
        const double t = sum + x;
        if (std::fabs(sum) >= std::fabs(x)) comp += (sum - t) + x;
        else comp += (x - t) + sum;
        sum = t;
      }
    }
    out[k] = (sum + comp) * dV;
  }
  return CLAW_OK;
}

struct CkptHeader {
  uint64_t magic;
  int64_t nx, ny;
  int32_t m, prec, scheme, pad;
};
static const uint64_t kMagic = 0x434c415743505431ull;

claw_status claw_checkpoint(claw_solver* s, void* host_buf, size_t* bytes) {
  if (!s || !s->bound || !bytes) return fail(s, "solver not bound");
  const size_t need = sizeof(CkptHeader) + sizeof(DevCtl) + s->sbytes;
  if (!host_buf) {
    *bytes = need;
    return CLAW_OK;
  }
  if (*bytes < need) return fail(s, "checkpoint buffer too small");
  SCK(enter(s));
  SCK(read_ctl(s));
  CkptHeader hd{kMagic, s->g.n[0], s->g.n[1], s->m.num_eqn, s->prec, s->m.scheme, 0};
  unsigned char* p = (unsigned char*)host_buf;
  std::memcpy(p, &hd, sizeof(hd));
  std::memcpy(p + sizeof(hd), s->h_ctl, sizeof(DevCtl));
  SCK(cudaMemcpyAsync(p + sizeof(hd) + sizeof(DevCtl), s->h_mem.q[s->h_ctl->cur], s->sbytes,
                      cudaMemcpyDeviceToHost, s->st));
  SCK(cudaStreamSynchronize(s->st));
  SCK(leave(s));
  *bytes = need;
  return CLAW_OK;
}

claw_status claw_restore(claw_solver* s, const void* host_buf, size_t bytes) {
  if (!s || !s->bound || !host_buf) return fail(s, "solver not bound");
  const size_t need = sizeof(CkptHeader) + sizeof(DevCtl) + s->sbytes;
  if (bytes < need) return fail(s, "checkpoint buffer too small");
  CkptHeader hd;
  std::memcpy(&hd, host_buf, sizeof(hd));
  if (hd.magic != kMagic || hd.nx != s->g.n[0] || hd.ny != s->g.n[1] || hd.m != s->m.num_eqn ||
      hd.prec != s->prec || hd.scheme != s->m.scheme)
    return fail(s, "checkpoint does not match this solver");
  DevCtl c;
  std::memcpy(&c, (const unsigned char*)host_buf + sizeof(hd), sizeof(DevCtl));
  c.cur = 0;
  c.nbuf = s->nbuf;
  c.accept_shift = make_ctl(s->m, s->g, s->nbuf, 0.0, 0.0).accept_shift;
  c.arrive = 0;
  c.smax[0] = c.smax[1] = 0;
  c.bad = 0;
  c.dry = 0;
  SCK(enter(s));
  SCK(cudaMemcpyAsync(s->q_user, (const unsigned char*)host_buf + sizeof(hd) + sizeof(DevCtl),
                      s->sbytes, cudaMemcpyHostToDevice, s->st));
  SCK(cudaMemcpyAsync(s->d_ctl, &c, sizeof(DevCtl), cudaMemcpyHostToDevice, s->st));
  SCK(cudaStreamSynchronize(s->st));
  SCK(leave(s));
  return CLAW_OK;
}

claw_status claw_step_host(claw_solver* s, const void* q_host_in, void* q_host_out, int n) {
  if (!s || !s->bound) return fail(s, "solver not bound");
  SCK(enter(s));
  SCK(cudaMemcpyAsync(s->q_user, q_host_in, s->sbytes, cudaMemcpyHostToDevice, s->st));
  SCK(launch_reset_cur(s->d_ctl, s->st));
  for (int i = 0; i < n; ++i) SCK(solver_attempt(s, s->st));
  // the slot that holds the result when every attempt is accepted; a device
  // copy moves the result there otherwise, so both reads queue behind the
  // attempts with one synchronisation at the end
  const int shift = make_ctl(s->m, s->g, s->nbuf, 0.0, 0.0).accept_shift;
  const int dst = (int)(((long long)(n > 0 ? n : 0) * shift) % s->nbuf);
  SCK(launch_select_copy(s->d_mem, s->d_ctl, dst, s->sbytes, s->st));
  SCK(cudaMemcpyAsync(q_host_out, s->h_mem.q[dst], s->sbytes, cudaMemcpyDeviceToHost, s->st));
  SCK(cudaMemcpyAsync(s->h_ctl, s->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s->st));
  SCK(cudaStreamSynchronize(s->st));
  SCK(leave(s));
  return s->h_ctl->status;
}

claw_status claw_solver_destroy(claw_solver* s) {
  if (!s) return CLAW_OK;
  if (s->st) cudaStreamSynchronize(s->st);
  free_bound(s);
  if (s->ev_a) cudaEventDestroy(s->ev_a);
  if (s->ev_b) cudaEventDestroy(s->ev_b);
  if (s->st && s->st != s->ustream) cudaStreamDestroy(s->st);
  delete s;
  return CLAW_OK;
}

}  // extern "C"

// ===========================================================================
// batches
// ===========================================================================
struct claw_batch {
  claw_method m;
  int nd = 1, prec = 0, nbuf = 2, n = 0;
  KernelSet ks{};
  std::vector<unsigned char> consts;
  std::vector<claw_grid> grids;
  std::vector<size_t> sbytes;
  cudaStream_t ustream = nullptr, st = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  void* work = nullptr;
  DevCtl* d_ctl = nullptr;
  DevCtl* h_ctl = nullptr;  // pinned, n
  Member* d_mem = nullptr;
  std::vector<Member> h_mem;
  Tile* d_tiles = nullptr;
  std::vector<Tile> h_tiles;
  int ntiles = 0;
  Tile* d_mtiles = nullptr;  // max-speed tiles
  int nmtiles = 0;
  int* d_count = nullptr;
  int* h_count = nullptr;
  int bw = 128, h = 32;
  int faces = 0;              // per-face classic path (capacity / media-aware transverse)
  void* work3 = nullptr;      // the members' face arrays, one allocation
  std::vector<size_t> work3_bytes;
  Tile* d_tile0 = nullptr;    // (member 0, t) for the source steps of one member at a time
  cudaGraphExec_t gexec = nullptr;
  int gk = 0;
  int bound = 0;
  std::string err;
};

namespace {

claw_status bfail(claw_batch* b, const char* what, cudaError_t e = cudaSuccess) {
  std::string msg = what;
  if (e != cudaSuccess) {
    msg += ": ";
    msg += cudaGetErrorString(e);
  }
  if (b) b->err = msg;
  g_err = msg;
  return e != cudaSuccess ? CLAW_ECUDA : CLAW_EINVAL;
}

#define BCK(call)                                      \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return bfail(b, #call, e_); \
  } while (0)

void batch_free(claw_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->gk = 0;
  if (b->work) cudaFree(b->work);
  if (b->work3) cudaFree(b->work3);
  b->work3 = nullptr;
  if (b->d_tile0) cudaFree(b->d_tile0);
  b->d_tile0 = nullptr;
  if (b->d_ctl) cudaFree(b->d_ctl);
  if (b->d_mem) cudaFree(b->d_mem);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_mtiles) cudaFree(b->d_mtiles);
  if (b->d_count) cudaFree(b->d_count);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  if (b->h_count) cudaFreeHost(b->h_count);
  b->work = nullptr;
  b->d_ctl = nullptr;
  b->d_mem = nullptr;
  b->d_tiles = nullptr;
  b->d_mtiles = nullptr;
  b->d_count = nullptr;
  b->h_ctl = nullptr;
  b->h_count = nullptr;
  b->bound = 0;
}

cudaError_t batch_attempt(claw_batch* b, cudaStream_t st) {
  if (b->nd == 3) {
    // sweeps and update of one 3D member at a time, each on its own face arrays
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < b->n && e == cudaSuccess; ++k) {
      const Member& mb = b->h_mem[k];
      LaunchArgs a{b->d_mem + k, nullptr, mb.ntiles, b->consts.data(), 0, 0, 0, st,
                   {mb.nx, mb.ny, mb.nz}, mb.work3, b->work3_bytes[k]};
      e = b->ks.classic(a);
    }
    return e;
  }
  if (b->faces) {
    // the per-face kernels take one member: sweeps and update member by member
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < b->n && e == cudaSuccess; ++k) {
      const Member& mb = b->h_mem[k];
      const int n3[3] = {mb.nx, mb.ny, 1};
      e = launch_attempt(b->ks, b->m, b->d_mem + k, nullptr, mb.ntiles, b->consts.data(), b->bw,
                         b->h, st, b->d_tile0, maxspeed_tiles(mb.nx, mb.ny), 1, n3, mb.work3,
                         b->work3_bytes[k]);
    }
    return e;
  }
  return launch_attempt(b->ks, b->m, b->d_mem, b->d_tiles, b->ntiles, b->consts.data(),
                        b->bw, b->h, st, b->d_mtiles, b->nmtiles, b->n);
}

}  // namespace

extern "C" {

claw_status claw_batch_create(const claw_method* m, const claw_grid* grids, int n, void* stream,
                              claw_batch** out) {
  if (!m || !grids || !out || n <= 0) return bfail(nullptr, "bad argument");
  *out = nullptr;
  const int nd = grids[0].ndim;
  const int faces = m->scheme == CLAW_CLASSIC && nd <= 2 &&
                    (m->capa_index >= 0 || (nd == 2 && m->rp == CLAW_RP_ACOUSTICS_VC));
  for (int k = 0; k < n; ++k) {
    if (const char* why = check_grid(grids[k], *m)) return bfail(nullptr, why);
    if (grids[k].ndim != nd) return bfail(nullptr, "all members need the same ndim");
  }
  if (const char* why = check_method(*m, nd)) return bfail(nullptr, why);
  KernelSet ks = kernels_for(m->rp, nd, m->prec);
  if (!ks.valid) return bfail(nullptr, "no kernels for this solver/dimension/precision");
  claw_batch* b = new claw_batch();
  b->m = *m;
  b->nd = nd;
  b->prec = m->prec;
  b->nbuf = nbuf_of(*m);
  b->n = n;
  b->ks = ks;
  b->faces = faces;
  b->bw = std::min(b->bw, ks.max_bw);
  default_shape(*m, nd, b->bw, b->h);
  b->consts = make_consts(*m);
  b->grids.assign(grids, grids + n);
  for (auto& g : b->grids)
    if (g.ndim == 1) g.n[1] = 1;
  b->ustream = (cudaStream_t)stream;
  cudaError_t e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_a, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_b, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    claw_status st = bfail(b, "stream creation", e);
    claw_batch_destroy(b);
    return st;
  }
  *out = b;
  return CLAW_OK;
}

claw_status claw_batch_bind(claw_batch* b, void* const* q, const void* const* aux,
                            const double* t_end) {
  if (!b || !q || !t_end) return bfail(b, "bad argument");
  if (b->m.num_aux > 0 && !aux) return bfail(b, "this solver needs aux fields");
  batch_free(b);
  const int n = b->n;
  b->sbytes.resize(n);
  size_t total = 0;
  for (int k = 0; k < n; ++k) {
    b->sbytes[k] = align256(state_bytes_of(b->m, b->grids[k]));
    total += b->sbytes[k] * (b->nbuf - 1 + pre_buffers(b->m));
  }
  BCK(cudaMalloc(&b->work, total));
  if (b->nd == 3) {
    size_t w3 = 0;
    b->work3_bytes.assign(n, 0);
    for (int k = 0; k < n; ++k) {
      const claw_grid& g = b->grids[k];
      b->work3_bytes[k] = align256(classic3d_work_bytes((int)g.n[0], (int)g.n[1], (int)g.n[2],
                                                        b->m.num_eqn, b->prec));
      w3 += b->work3_bytes[k];
    }
    BCK(cudaMalloc(&b->work3, w3));
  }
  if (b->faces) {
    size_t w3 = 0;
    b->work3_bytes.assign(n, 0);
    for (int k = 0; k < n; ++k) {
      b->work3_bytes[k] = align256(faces_work_bytes(b->nd, (int)b->grids[k].n[0],
                                                    (int)b->grids[k].n[1], b->m.num_eqn, b->prec));
      w3 += b->work3_bytes[k];
    }
    BCK(cudaMalloc(&b->work3, w3));
    if (b->m.source != CLAW_SOURCE_NONE) {
      int most = 1;
      for (int k = 0; k < n; ++k)
        most = std::max(most, maxspeed_tiles((int)b->grids[k].n[0], (int)b->grids[k].n[1]));
      std::vector<Tile> t0(most);
      for (int t = 0; t < most; ++t) t0[t] = Tile{0, t};
      BCK(cudaMalloc(&b->d_tile0, sizeof(Tile) * most));
      BCK(cudaMemcpy(b->d_tile0, t0.data(), sizeof(Tile) * most, cudaMemcpyHostToDevice));
    }
  }
  BCK(cudaMalloc(&b->d_ctl, sizeof(DevCtl) * n));
  BCK(cudaMalloc(&b->d_mem, sizeof(Member) * n));
  BCK(cudaMallocHost(&b->h_ctl, sizeof(DevCtl) * n));
  BCK(cudaMalloc(&b->d_count, sizeof(int)));
  BCK(cudaMallocHost(&b->h_count, sizeof(int)));
  b->h_mem.assign(n, Member{});
  b->h_tiles.clear();
  std::vector<Tile> mt;
  unsigned char* w = (unsigned char*)b->work;
  unsigned char* w3p = (unsigned char*)b->work3;
  for (int k = 0; k < n; ++k) {
    const claw_grid& g = b->grids[k];
    Member& mb = b->h_mem[k];
    mb.q[0] = q[k];
    for (int j = 1; j < b->nbuf; ++j) {
      mb.q[j] = w;
      w += b->sbytes[k];
    }
    if (pre_buffers(b->m)) {
      mb.qpre = w;
      w += b->sbytes[k];
    }
    mb.aux = aux ? aux[k] : nullptr;
    mb.nx = (int)g.n[0];
    mb.ny = (int)g.n[1];
    mb.nz = 1;
    mb.ctl = b->d_ctl + k;
    if (b->nd == 3) {
      // the 3D kernels take one member; the update's blocks count the arrivals
      mb.nz = (int)g.n[2];
      mb.ntiles = classic3d_update_blocks(cells_of(g));
      mb.work3 = w3p;
      w3p += b->work3_bytes[k];
    } else if (b->faces) {
      // the update's blocks (256 cells each) count the arrivals
      mb.ntiles = (int)((cells_of(g) + 255) / 256);
      mb.work3 = w3p;
      w3p += b->work3_bytes[k];
    } else {
      mb.ntiles = tiles_of(b->m.scheme, b->nd, b->prec, b->ks.MA, mb.nx, mb.ny, b->bw, b->h);
      for (int t = 0; t < mb.ntiles; ++t) b->h_tiles.push_back(Tile{k, t});
    }
    const int ms = b->nd == 3 ? 0 : maxspeed_tiles(mb.nx, mb.ny);
    for (int t = 0; t < ms; ++t) mt.push_back(Tile{k, t});
    b->h_ctl[k] = make_ctl(b->m, g, b->nbuf, 0.0, t_end[k]);
  }
  b->ntiles = (int)b->h_tiles.size();
  b->nmtiles = (int)mt.size();
  BCK(cudaMalloc(&b->d_tiles, sizeof(Tile) * std::max(b->ntiles, 1)));
  BCK(cudaMalloc(&b->d_mtiles, sizeof(Tile) * std::max(b->nmtiles, 1)));
  BCK(cudaEventRecord(b->ev_a, b->ustream));
  BCK(cudaStreamWaitEvent(b->st, b->ev_a, 0));
  BCK(cudaMemcpyAsync(b->d_ctl, b->h_ctl, sizeof(DevCtl) * n, cudaMemcpyHostToDevice, b->st));
  BCK(cudaMemcpyAsync(b->d_mem, b->h_mem.data(), sizeof(Member) * n, cudaMemcpyHostToDevice, b->st));
  if (b->ntiles > 0)
    BCK(cudaMemcpyAsync(b->d_tiles, b->h_tiles.data(), sizeof(Tile) * b->ntiles,
                        cudaMemcpyHostToDevice, b->st));
  if (b->nmtiles > 0)
    BCK(cudaMemcpyAsync(b->d_mtiles, mt.data(), sizeof(Tile) * b->nmtiles,
                        cudaMemcpyHostToDevice, b->st));
  if (b->nd == 3) {
    for (int k = 0; k < n; ++k) {
      const claw_grid& g = b->grids[k];
      LaunchArgs a{b->d_mem + k, nullptr, 0, b->consts.data(), 0, 0, 0, b->st,
                   {(int)g.n[0], (int)g.n[1], (int)g.n[2]}, nullptr, 0};
      BCK(b->ks.maxspeed(a));
    }
  } else {
    LaunchArgs a{b->d_mem, b->d_mtiles, b->nmtiles, b->consts.data(), 0, 0, 0, b->st};
    BCK(b->ks.maxspeed(a));
  }
  BCK(launch_dt_init(b->d_ctl, n, b->st));
  BCK(cudaStreamSynchronize(b->st));
  b->bound = 1;
  return CLAW_OK;
}

claw_status claw_batch_advance(claw_batch* b, int n) {
  if (!b || !b->bound) return bfail(b, "batch not bound");
  BCK(cudaEventRecord(b->ev_a, b->ustream));
  BCK(cudaStreamWaitEvent(b->st, b->ev_a, 0));
  for (int i = 0; i < n; ++i) BCK(batch_attempt(b, b->st));
  BCK(cudaEventRecord(b->ev_b, b->st));
  BCK(cudaStreamWaitEvent(b->ustream, b->ev_b, 0));
  return CLAW_OK;
}

claw_status claw_batch_info(claw_batch* b, claw_step_info* info) {
  if (!b || !b->bound) return bfail(b, "batch not bound");
  BCK(cudaEventRecord(b->ev_a, b->ustream));
  BCK(cudaStreamWaitEvent(b->st, b->ev_a, 0));
  BCK(cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(DevCtl) * b->n, cudaMemcpyDeviceToHost, b->st));
  BCK(cudaStreamSynchronize(b->st));
  if (info)
    for (int k = 0; k < b->n; ++k) fill_info(b->h_ctl[k], info + k);
  return CLAW_OK;
}

claw_status claw_batch_sync_state(claw_batch* b) {
  if (!b || !b->bound) return bfail(b, "batch not bound");
  BCK(cudaEventRecord(b->ev_a, b->ustream));
  BCK(cudaStreamWaitEvent(b->st, b->ev_a, 0));
  BCK(cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(DevCtl) * b->n, cudaMemcpyDeviceToHost, b->st));
  BCK(cudaStreamSynchronize(b->st));
  bool any = false;
  for (int k = 0; k < b->n; ++k) {
    const int cur = b->h_ctl[k].cur;
    if (cur != 0) {
      any = true;
      BCK(cudaMemcpyAsync(b->h_mem[k].q[0], b->h_mem[k].q[cur],
                          state_bytes_of(b->m, b->grids[k]), cudaMemcpyDeviceToDevice, b->st));
      BCK(launch_reset_cur(b->d_ctl + k, b->st));
    }
  }
  if (any) BCK(cudaStreamSynchronize(b->st));
  BCK(cudaEventRecord(b->ev_b, b->st));
  BCK(cudaStreamWaitEvent(b->ustream, b->ev_b, 0));
  return CLAW_OK;
}

claw_status claw_batch_evolve(claw_batch* b, int use_graph, int64_t max_steps,
                              claw_step_info* info) {
  if (!b || !b->bound) return bfail(b, "batch not bound");
  BCK(cudaEventRecord(b->ev_a, b->ustream));
  BCK(cudaStreamWaitEvent(b->st, b->ev_a, 0));
  if (max_steps > 0) {
    // per-member step limit on top of each member's own t_end
    BCK(cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(DevCtl) * b->n, cudaMemcpyDeviceToHost, b->st));
    BCK(cudaStreamSynchronize(b->st));
    for (int k = 0; k < b->n; ++k) b->h_ctl[k].max_steps = b->h_ctl[k].steps + max_steps;
    BCK(cudaMemcpyAsync(b->d_ctl, b->h_ctl, sizeof(DevCtl) * b->n, cudaMemcpyHostToDevice, b->st));
  }
  const int GK = 16;
  if (use_graph && b->gk != GK) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < GK && e == cudaSuccess; ++i) e = batch_attempt(b, b->st);
    cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
    if (e != cudaSuccess) return bfail(b, "graph capture", e);
    if (e2 != cudaSuccess) return bfail(b, "graph capture", e2);
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, "graph instantiate", e);
    b->gk = GK;
  }
  long long launched = 0;
  for (;;) {
    BCK(launch_count_active(b->d_ctl, b->n, b->d_count, b->st));
    BCK(cudaMemcpyAsync(b->h_count, b->d_count, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    BCK(cudaStreamSynchronize(b->st));
    if (*b->h_count == 0) break;
    for (int r = 0; r < 4; ++r) {
      if (use_graph) BCK(cudaGraphLaunch(b->gexec, b->st));
      else
        for (int i = 0; i < GK; ++i) BCK(batch_attempt(b, b->st));
    }
    launched += 4 * GK;
    if (launched > (1LL << 40)) return bfail(b, "batch made no progress");
  }
  BCK(cudaEventRecord(b->ev_b, b->st));
  BCK(cudaStreamWaitEvent(b->ustream, b->ev_b, 0));
  claw_status st = claw_batch_sync_state(b);
  if (st != CLAW_OK) return st;
  claw_status worst = CLAW_OK;
  for (int k = 0; k < b->n; ++k) {
    if (info) fill_info(b->h_ctl[k], info + k);
    if (b->h_ctl[k].status != CLAW_OK) worst = b->h_ctl[k].status;
  }
  return worst;
}

claw_status claw_batch_tune(claw_batch* b, int mode, int* bw, int* h) {
  if (!b || !b->bound) return bfail(b, "batch not bound");
  const bool tunable = !b->faces && b->nd <= 2;
  if (tunable) {
    int nbw = b->bw, nh = b->h;
    if (mode == 0) {
      BCK(cudaEventRecord(b->ev_a, b->ustream));
      BCK(cudaStreamWaitEvent(b->st, b->ev_a, 0));
      BCK(tune_members(b->ks, b->nd, b->m, b->h_mem, b->consts.data(), b->st, nbw, nh));
    } else {
      if (!bw || !h) return bfail(b, "bad tile shape");
      const int want_bw = (b->m.scheme == CLAW_CLASSIC && b->nd == 1) ? b->bw : *bw;
      if (const char* why = bad_shape(b->ks, b->m, b->nd, want_bw, *h))
        return bfail(b, why);
      nbw = want_bw;
      nh = *h;
    }
    b->bw = nbw;
    b->h = nh;
    // the tile table and the members' tile counts for the new shape
    b->h_tiles.clear();
    for (int k = 0; k < b->n; ++k) {
      Member& mb = b->h_mem[k];
      mb.ntiles = tiles_of(b->m.scheme, b->nd, b->prec, b->ks.MA, mb.nx, mb.ny, b->bw, b->h);
      for (int t = 0; t < mb.ntiles; ++t) b->h_tiles.push_back(Tile{k, t});
    }
    if ((int)b->h_tiles.size() > b->ntiles) {
      BCK(cudaStreamSynchronize(b->st));
      BCK(cudaFree(b->d_tiles));
      b->d_tiles = nullptr;
      BCK(cudaMalloc(&b->d_tiles, sizeof(Tile) * b->h_tiles.size()));
    }
    b->ntiles = (int)b->h_tiles.size();
    BCK(cudaMemcpyAsync(b->d_mem, b->h_mem.data(), sizeof(Member) * b->n,
                        cudaMemcpyHostToDevice, b->st));
    BCK(cudaMemcpyAsync(b->d_tiles, b->h_tiles.data(), sizeof(Tile) * b->ntiles,
                        cudaMemcpyHostToDevice, b->st));
    BCK(cudaStreamSynchronize(b->st));
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->gk = 0;
  }
  if (bw) *bw = b->bw;
  if (h) *h = b->h;
  return CLAW_OK;
}

claw_status claw_batch_destroy(claw_batch* b) {
  if (!b) return CLAW_OK;
  if (b->st) cudaStreamSynchronize(b->st);
  batch_free(b);
  if (b->ev_a) cudaEventDestroy(b->ev_a);
  if (b->ev_b) cudaEventDestroy(b->ev_b);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
  return CLAW_OK;
}

}  // extern "C"

// ===========================================================================
// serving: continuous batching
// ===========================================================================
namespace {
struct Req {
  uint64_t ticket = 0;
  claw_grid g{};
  std::vector<unsigned char> q0, aux0, result;
  double t_end = 0;
  int status = CLAW_EBUSY;
  double t_submit = 0, t_admit = 0, t_done = 0, t_reached = 0;
  long long steps = 0;
  void* dblock = nullptr;
  size_t dbytes = 0;
  size_t w3bytes = 0;  // per-face path: the request's face arrays
  Member mem{};
  double rem = -1.0;   // estimated cell updates left (< 0: not stepped yet)
  int idle = 0;        // pumps in a row this request was left out of
};
}  // namespace

struct claw_server {
  claw_method m;
  int prec = 0, nbuf = 2, nd = 2;
  KernelSet ks{};
  std::vector<unsigned char> consts;
  size_t budget = 0, used = 0;
  int max_slots = 0;
  cudaStream_t ustream = nullptr, st = nullptr;
  uint64_t next_ticket = 1;
  std::deque<uint64_t> queue;
  std::vector<uint64_t> running;
  std::map<uint64_t, Req> reqs;
  Member* d_mem = nullptr;
  Tile* d_tiles = nullptr;
  Tile* d_stiles = nullptr;  // cell tiles of the source step (methods with a source)
  size_t cap_mem = 0, cap_tiles = 0, cap_stiles = 0;
  int ntiles = 0, nstiles = 0;
  bool dirty = true;
  DevCtl* d_gather = nullptr;
  DevCtl* h_gather = nullptr;  // pinned, two halves of max_slots (one per pump parity)
  // pipelined pumps: the statuses gathered after the last pump's attempts
  cudaStream_t cst = nullptr;  // result copies of finished requests
  cudaEvent_t ev_gather[2] = {nullptr, nullptr}, ev_copy = nullptr;
  bool gather_pending = false;
  int gpar = 0;                          // parity of the next gather
  std::vector<uint64_t> gathered;        // the requests of the pending gather
  std::vector<char> gathered_stepped;    // ... and whether that pump stepped them
  // pinned staging of a pump's uploads (copies from pageable memory would
  // wait for the stream's queued attempts); reused by the next pump after
  // ev_stage
  unsigned char* stage = nullptr;
  size_t stage_cap = 0, stage_off = 0;
  cudaEvent_t ev_stage = nullptr;
  bool stage_used = false;
  // 2D classic tile for every request: the shape the autotuner picks for a
  // 1024 x 1024 FP32 grid, and the fastest of those tried on a mixed stream
  int bw = 64, h = 21;
  int faces = 0;  // per-face classic path: kernels run request by request
  Tile* d_tile0 = nullptr;  // (member 0, t): source steps of one request at a time
  size_t cap_tile0 = 0;
  // scheduling: the requests the step tables cover (d_smem, d_tiles, d_stiles)
  int sched = CLAW_SCHED_SRW;
  long long sched_cells = 1LL << 23;
  std::vector<uint64_t> sel;
  Member* d_smem = nullptr;
  size_t cap_smem = 0;
  std::deque<uint64_t> completed;  // finished, not yet handed out by take_done
  std::string err;
};

namespace {

claw_status sfail(claw_server* v, const char* what, cudaError_t e = cudaSuccess) {
  std::string msg = what;
  if (e != cudaSuccess) {
    msg += ": ";
    msg += cudaGetErrorString(e);
  }
  if (v) v->err = msg;
  g_err = msg;
  return e != cudaSuccess ? CLAW_ECUDA : CLAW_EINVAL;
}

#define VCK(call)                                      \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return sfail(v, #call, e_); \
  } while (0)

size_t req_faces_bytes(const claw_server* v, const claw_grid& g) {
  if (v->nd == 3)
    return align256(classic3d_work_bytes((int)g.n[0], (int)g.n[1], (int)g.n[2], v->m.num_eqn,
                                         v->prec));
  return v->faces ? align256(faces_work_bytes(v->nd, (int)g.n[0], (int)g.n[1], v->m.num_eqn,
                                              v->prec))
                  : 0;
}

size_t req_bytes(const claw_server* v, const claw_grid& g) {
  return align256(state_bytes_of(v->m, g)) * (v->nbuf + pre_buffers(v->m)) +
         align256(aux_bytes_of(v->m, g)) + align256(sizeof(DevCtl)) + req_faces_bytes(v, g);
}

}  // namespace

extern "C" {

double claw_clock(void) { return now_s(); }

claw_status claw_server_create_nd(const claw_method* m, int ndim, size_t hbm_budget_bytes,
                                  int max_slots, void* stream, claw_server** out) {
  if (!m || !out || max_slots <= 0 || ndim < 1 || ndim > 3) return sfail(nullptr, "bad argument");
  *out = nullptr;
  const int nd = ndim;
  if (const char* why = check_method(*m, nd)) return sfail(nullptr, why);
  const int faces = m->scheme == CLAW_CLASSIC && nd <= 2 &&
                    (m->capa_index >= 0 || (nd == 2 && m->rp == CLAW_RP_ACOUSTICS_VC));
  KernelSet ks = kernels_for(m->rp, nd, m->prec);
  if (!ks.valid) return sfail(nullptr, "no kernels for this solver/dimension/precision");
  claw_server* v = new claw_server();
  v->m = *m;
  v->prec = m->prec;
  v->nd = nd;
  v->nbuf = nbuf_of(*m);
  v->ks = ks;
  v->faces = faces;
  v->bw = std::min(v->bw, ks.max_bw);
  default_shape(*m, nd, v->bw, v->h);
  v->consts = make_consts(*m);
  v->budget = hbm_budget_bytes;
  v->max_slots = max_slots;
  v->ustream = (cudaStream_t)stream;
  cudaError_t e = cudaStreamCreateWithFlags(&v->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&v->cst, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&v->ev_gather[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->ev_copy, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->ev_stage, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&v->d_gather, sizeof(DevCtl) * max_slots);
  if (e == cudaSuccess) e = cudaMallocHost(&v->h_gather, 2 * sizeof(DevCtl) * max_slots);
  if (e == cudaSuccess) {
    cudaMemPool_t pool;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  if (e != cudaSuccess) {
    claw_status st = sfail(v, "server setup", e);
    claw_server_destroy(v);
    return st;
  }
  *out = v;
  return CLAW_OK;
}

claw_status claw_server_create(const claw_method* m, size_t hbm_budget_bytes, int max_slots,
                               void* stream, claw_server** out) {
  if (!m) return sfail(nullptr, "bad argument");
  // the dimension from the number of fields: 2D when it matches the 2D system
  const int nd = (m->num_eqn == num_eqn(m->rp, 2)) ? 2 : 1;
  return claw_server_create_nd(m, nd, hbm_budget_bytes, max_slots, stream, out);
}

claw_status claw_server_submit(claw_server* v, const claw_grid* g, const void* q0_host,
                               const void* aux_host, double t_end, uint64_t* ticket) {
  if (!v || !g || !q0_host || !ticket) return sfail(v, "bad argument");
  if (g->ndim != v->nd) return sfail(v, "grid dimension does not match the server's method");
  if (const char* why = check_grid(*g, v->m)) return sfail(v, why);
  if (v->m.num_aux > 0 && !aux_host) return sfail(v, "this solver needs aux fields");
  Req r;
  r.ticket = v->next_ticket++;
  r.g = *g;
  if (r.g.ndim == 1) r.g.n[1] = 1;
  r.dbytes = req_bytes(v, r.g);
  if (r.dbytes > v->budget) {
    g_err = v->err = "request exceeds the HBM budget";
    return CLAW_EBUDGET;
  }
  const size_t sb = state_bytes_of(v->m, r.g), ab = aux_bytes_of(v->m, r.g);
  r.q0.assign((const unsigned char*)q0_host, (const unsigned char*)q0_host + sb);
  if (ab) r.aux0.assign((const unsigned char*)aux_host, (const unsigned char*)aux_host + ab);
  r.t_end = t_end;
  r.t_submit = now_s();
  *ticket = r.ticket;
  v->queue.push_back(r.ticket);
  v->reqs.emplace(r.ticket, std::move(r));
  return CLAW_OK;
}

namespace {
// Upload n bytes from host memory to dst on the server's stream through the
// pinned staging buffer (the host copy is immediate; the transfer runs in
// stream order).  Growing the buffer waits for the stream (the transfers
// already queued from the old one) first.
cudaError_t stage_upload(claw_server* v, void* dst, const void* src, size_t n) {
  if (n == 0) return cudaSuccess;
  size_t off = (v->stage_off + 255) & ~(size_t)255;
  if (off + n > v->stage_cap) {
    cudaError_t e = cudaStreamSynchronize(v->st);
    if (e != cudaSuccess) return e;
    if (v->stage) cudaFreeHost(v->stage);
    v->stage = nullptr;
    v->stage_cap = std::max<size_t>({2 * v->stage_cap, n + 256, (size_t)16 << 20});
    if ((e = cudaMallocHost(&v->stage, v->stage_cap)) != cudaSuccess) {
      v->stage_cap = 0;
      return e;
    }
    off = 0;
  }
  std::memcpy(v->stage + off, src, n);
  v->stage_off = off + n;
  return cudaMemcpyAsync(dst, v->stage + off, n, cudaMemcpyHostToDevice, v->st);
}
}  // namespace

claw_status claw_server_pump(claw_server* v, int steps, int* running, int* queued) {
  if (!v) return sfail(nullptr, "null server");
  // The pump is pipelined: its attempts are enqueued first, then the host
  // reads the statuses the previous pump gathered, retires, admits and
  // chooses the next pump's requests while the GPU runs them.  A request is
  // therefore stepped from the pump after the one that admitted it, and
  // handed out by the pump after the one whose attempts finished it.
  // 1. this pump's attempts, over the step tables chosen at the end of the
  // previous pump (requests that finished since are skipped by the kernels,
  // their control blocks say done): the GPU runs them while the host does
  // the bookkeeping below
  std::vector<uint64_t> launched = v->sel;
  if (!v->sel.empty()) {
    for (int i = 0; i < steps; ++i) {
      if (v->nd == 3) {
        // the 3D sweeps take one member: request by request
        for (size_t k = 0; k < v->sel.size(); ++k) {
          const Req& r = v->reqs[v->sel[k]];
          LaunchArgs a{v->d_smem + k, nullptr, r.mem.ntiles, v->consts.data(), 0, 0, 0, v->st,
                       {r.mem.nx, r.mem.ny, r.mem.nz}, r.mem.work3, r.w3bytes};
          VCK(v->ks.classic(a));
        }
      } else if (v->faces) {
        // the per-face kernels take one member: request by request
        for (size_t k = 0; k < v->sel.size(); ++k) {
          const Req& r = v->reqs[v->sel[k]];
          const int n3[3] = {r.mem.nx, r.mem.ny, 1};
          VCK(launch_attempt(v->ks, v->m, v->d_smem + k, nullptr, r.mem.ntiles,
                             v->consts.data(), v->bw, v->h, v->st, v->d_tile0,
                             maxspeed_tiles(r.mem.nx, r.mem.ny), 1, n3, r.mem.work3,
                             r.w3bytes));
        }
      } else {
        VCK(launch_attempt(v->ks, v->m, v->d_smem, v->d_tiles, v->ntiles, v->consts.data(),
                           v->bw, v->h, v->st, v->d_stiles, v->nstiles, (int)v->sel.size()));
      }
    }
  }
  // 2. the previous pump's statuses, gathered after its attempts: retire
  // finished requests (their results copied on the copy stream once those
  // attempts are done, their memory freed after the copies), update the
  // remaining-work estimates
  if (v->gather_pending) {
    const int g = v->gpar ^ 1;  // parity of the pending gather
    VCK(cudaEventSynchronize(v->ev_gather[g]));
    v->gather_pending = false;
    const std::vector<uint64_t>& gt = v->gathered;
    std::vector<char> fin(gt.size(), 0);
    bool any_fin = false;
    for (size_t i = 0; i < gt.size(); ++i) {
      Req& r = v->reqs[gt[i]];
      const DevCtl& c = v->h_gather[g * v->max_slots + i];
      r.steps = c.steps;
      r.t_reached = c.t;
      const double cells = (double)cells_of(r.g);
      r.rem = (c.dt > 0.0 && c.t < r.t_end) ? cells * std::ceil((r.t_end - c.t) / c.dt) : cells;
      r.idle = v->gathered_stepped[i] ? 0 : r.idle + 1;
      if (c.done) {
        if (!any_fin) VCK(cudaStreamWaitEvent(v->cst, v->ev_gather[g], 0));
        any_fin = true;
        const size_t sb = state_bytes_of(v->m, r.g);
        r.result.resize(sb);
        VCK(cudaMemcpyAsync(r.result.data(), r.mem.q[c.cur], sb, cudaMemcpyDeviceToHost, v->cst));
        r.status = c.status;
        fin[i] = 1;
      }
    }
    if (any_fin) {
      VCK(cudaStreamSynchronize(v->cst));
      VCK(cudaEventRecord(v->ev_copy, v->cst));
      VCK(cudaStreamWaitEvent(v->st, v->ev_copy, 0));
      const double now = now_s();
      std::vector<uint64_t> keep;
      for (uint64_t t : v->running) {
        const auto it = std::find(gt.begin(), gt.end(), t);
        if (it != gt.end() && fin[it - gt.begin()]) {
          Req& r = v->reqs[t];
          r.t_done = now;
          v->completed.push_back(r.ticket);
          VCK(cudaFreeAsync(r.dblock, v->st));
          r.dblock = nullptr;
          v->used -= r.dbytes;
          v->dirty = true;
        } else {
          keep.push_back(t);
        }
      }
      v->running.swap(keep);
    }
  }
  // 3. admission: first-come first-served while the budget and slots allow
  if (v->stage_used) {  // the last pump's uploads are done before their staging is reused
    VCK(cudaEventSynchronize(v->ev_stage));
    v->stage_used = false;
  }
  v->stage_off = 0;
  std::vector<uint64_t> admitted;
  while (!v->queue.empty() && (int)v->running.size() < v->max_slots) {
    Req& r = v->reqs[v->queue.front()];
    if (v->used + r.dbytes > v->budget) break;
    VCK(cudaMallocAsync(&r.dblock, r.dbytes, v->st));
    v->used += r.dbytes;
    const size_t sb = align256(state_bytes_of(v->m, r.g));
    unsigned char* p = (unsigned char*)r.dblock;
    std::memset(&r.mem, 0, sizeof(Member));
    for (int j = 0; j < v->nbuf; ++j) r.mem.q[j] = p + j * sb;
    p += sb * v->nbuf;
    if (pre_buffers(v->m)) {  // Strang: Q^n after the first half source step
      r.mem.qpre = p;
      p += sb;
    }
    const size_t ab = align256(aux_bytes_of(v->m, r.g));
    r.mem.aux = ab ? p : nullptr;
    p += ab;
    r.mem.ctl = (DevCtl*)p;
    p += align256(sizeof(DevCtl));
    r.mem.nx = (int)r.g.n[0];
    r.mem.ny = (int)r.g.n[1];
    r.mem.nz = v->nd == 3 ? (int)r.g.n[2] : 1;
    if (v->faces || v->nd == 3) {
      // face arrays; the update's blocks (256 cells each) count the arrivals
      r.w3bytes = req_faces_bytes(v, r.g);
      r.mem.work3 = p;
      r.mem.ntiles = v->nd == 3 ? classic3d_update_blocks(cells_of(r.g))
                                : (int)((cells_of(r.g) + 255) / 256);
    } else {
      r.mem.ntiles =
          tiles_of(v->m.scheme, v->nd, v->prec, v->ks.MA, r.mem.nx, r.mem.ny, v->bw, v->h);
    }
    DevCtl c = make_ctl(v->m, r.g, v->nbuf, 0.0, r.t_end);
    VCK(stage_upload(v, r.mem.q[0], r.q0.data(), r.q0.size()));
    if (!r.aux0.empty()) VCK(stage_upload(v, (void*)r.mem.aux, r.aux0.data(), r.aux0.size()));
    VCK(stage_upload(v, r.mem.ctl, &c, sizeof(DevCtl)));
    r.t_admit = now_s();
    admitted.push_back(r.ticket);
    v->running.push_back(r.ticket);
    v->queue.pop_front();
    v->dirty = true;
  }
  // 4. rebuild the member table of the running requests when the set changed
  if (v->dirty) {
    std::vector<Member> hm;
    for (uint64_t t : v->running) hm.push_back(v->reqs[t].mem);
    if (hm.size() > v->cap_mem) {
      if (v->d_mem) VCK(cudaFreeAsync(v->d_mem, v->st));
      v->cap_mem = std::max<size_t>(hm.size(), 2 * v->cap_mem);
      VCK(cudaMallocAsync(&v->d_mem, sizeof(Member) * v->cap_mem, v->st));
    }
    if (!hm.empty())
      VCK(stage_upload(v, v->d_mem, hm.data(), sizeof(Member) * hm.size()));
    if (v->faces && v->m.source != CLAW_SOURCE_NONE) {
      size_t most = 1;
      for (uint64_t t : v->running) {
        const Req& r = v->reqs[t];
        most = std::max<size_t>(most, (size_t)maxspeed_tiles(r.mem.nx, r.mem.ny));
      }
      if (most > v->cap_tile0) {
        if (v->d_tile0) VCK(cudaFreeAsync(v->d_tile0, v->st));
        v->cap_tile0 = std::max(most, 2 * v->cap_tile0);
        std::vector<Tile> t0(v->cap_tile0);
        for (size_t t = 0; t < v->cap_tile0; ++t) t0[t] = Tile{0, (int)t};
        VCK(cudaMallocAsync(&v->d_tile0, sizeof(Tile) * v->cap_tile0, v->st));
        VCK(cudaMemcpyAsync(v->d_tile0, t0.data(), sizeof(Tile) * v->cap_tile0,
                            cudaMemcpyHostToDevice, v->st));
        VCK(cudaStreamSynchronize(v->st));  // t0 is a host temporary
      }
    }
    // first dt for the newly admitted requests
    if (!admitted.empty() && v->nd == 3) {
      for (size_t i = 0; i < v->running.size(); ++i) {
        const Req& r = v->reqs[v->running[i]];
        if (std::find(admitted.begin(), admitted.end(), r.ticket) == admitted.end()) continue;
        LaunchArgs a{v->d_mem + i, nullptr, 0, v->consts.data(), 0, 0, 0, v->st,
                     {r.mem.nx, r.mem.ny, r.mem.nz}, nullptr, 0};
        VCK(v->ks.maxspeed(a));
      }
      for (uint64_t t : admitted) VCK(launch_dt_init(v->reqs[t].mem.ctl, 1, v->st));
    } else if (!admitted.empty()) {
      std::vector<Tile> ms;
      for (size_t i = 0; i < v->running.size(); ++i) {
        const Req& r = v->reqs[v->running[i]];
        if (std::find(admitted.begin(), admitted.end(), r.ticket) == admitted.end()) continue;
        const int n = maxspeed_tiles(r.mem.nx, r.mem.ny);
        for (int t = 0; t < n; ++t) ms.push_back(Tile{(int)i, t});
      }
      Tile* d_ms = nullptr;
      VCK(cudaMallocAsync(&d_ms, sizeof(Tile) * ms.size(), v->st));
      VCK(stage_upload(v, d_ms, ms.data(), sizeof(Tile) * ms.size()));
      LaunchArgs a{v->d_mem, d_ms, (int)ms.size(), v->consts.data(), 0, 0, 0, v->st};
      VCK(v->ks.maxspeed(a));
      for (uint64_t t : admitted) VCK(launch_dt_init(v->reqs[t].mem.ctl, 1, v->st));
      VCK(cudaFreeAsync(d_ms, v->st));
    }
    v->dirty = false;
  }
  // 5. choose the requests the next pump steps (every running one, or the
  // least remaining work first until sched_cells cells are covered) and
  // rebuild the step tables when the choice changed (stream-ordered after
  // this pump's attempts, which read the old ones)
  if (v->running.empty()) {
    v->sel.clear();
  } else {
    std::vector<uint64_t> sel;
    if (v->sched == CLAW_SCHED_ALL) {
      sel = v->running;
    } else {
      // not yet stepped first, then requests left out of kStarve pumps, then
      // by remaining work; ties by ticket (arrival order)
      constexpr int kStarve = 16;
      const int nr = (int)v->running.size();
      std::vector<std::tuple<int, double, uint64_t, int>> order(nr);
      for (int i = 0; i < nr; ++i) {
        const uint64_t t = v->running[i];
        const Req& r = v->reqs[t];
        const int cls = r.rem < 0 ? 0 : (r.idle >= kStarve ? 1 : 2);
        order[i] = std::make_tuple(cls, cls == 2 ? r.rem : 0.0, t, i);
      }
      std::sort(order.begin(), order.end());
      std::vector<int> picked;
      long long cells = 0;
      for (const auto& o : order) {
        const Req& r = v->reqs[std::get<2>(o)];
        if (cells >= v->sched_cells && std::get<0>(o) == 2) continue;
        picked.push_back(std::get<3>(o));
        cells += (long long)cells_of(r.g);
      }
      // keep the member order of the running list (tile tables stay stable)
      std::sort(picked.begin(), picked.end());
      for (int i : picked) sel.push_back(v->running[i]);
    }
    if (sel != v->sel) {
      std::vector<Member> hm;
      std::vector<Tile> ht, hs;
      for (size_t i = 0; i < sel.size(); ++i) {
        const Req& r = v->reqs[sel[i]];
        hm.push_back(r.mem);
        if (!v->faces && v->nd != 3)
          for (int t = 0; t < r.mem.ntiles; ++t) ht.push_back(Tile{(int)i, t});
        if (v->m.source != CLAW_SOURCE_NONE)
          for (int t = 0; t < maxspeed_tiles(r.mem.nx, r.mem.ny); ++t) hs.push_back(Tile{(int)i, t});
      }
      if (hm.size() > v->cap_smem) {
        if (v->d_smem) VCK(cudaFreeAsync(v->d_smem, v->st));
        v->cap_smem = std::max<size_t>(hm.size(), 2 * v->cap_smem);
        VCK(cudaMallocAsync(&v->d_smem, sizeof(Member) * v->cap_smem, v->st));
      }
      VCK(stage_upload(v, v->d_smem, hm.data(), sizeof(Member) * hm.size()));
      if (ht.size() > v->cap_tiles) {
        if (v->d_tiles) VCK(cudaFreeAsync(v->d_tiles, v->st));
        v->cap_tiles = std::max<size_t>(ht.size(), 2 * v->cap_tiles);
        VCK(cudaMallocAsync(&v->d_tiles, sizeof(Tile) * v->cap_tiles, v->st));
      }
      if (!ht.empty())
        VCK(stage_upload(v, v->d_tiles, ht.data(), sizeof(Tile) * ht.size()));
      v->ntiles = (int)ht.size();
      if (hs.size() > v->cap_stiles) {
        if (v->d_stiles) VCK(cudaFreeAsync(v->d_stiles, v->st));
        v->cap_stiles = std::max<size_t>(hs.size(), 2 * v->cap_stiles);
        VCK(cudaMallocAsync(&v->d_stiles, sizeof(Tile) * v->cap_stiles, v->st));
      }
      if (!hs.empty())
        VCK(stage_upload(v, v->d_stiles, hs.data(), sizeof(Tile) * hs.size()));
      v->nstiles = (int)hs.size();
      v->sel = sel;
    }
  }
  if (v->stage_off > 0) {
    VCK(cudaEventRecord(v->ev_stage, v->st));
    v->stage_used = true;
  }
  // 6. gather the statuses of the running requests after this pump's
  // attempts (read by the next pump)
  if (!v->running.empty()) {
    const int cnt = (int)v->running.size();
    VCK(launch_gather_ctl(v->d_mem, cnt, v->d_gather, v->st));
    VCK(cudaMemcpyAsync(v->h_gather + v->gpar * v->max_slots, v->d_gather, sizeof(DevCtl) * cnt,
                        cudaMemcpyDeviceToHost, v->st));
    VCK(cudaEventRecord(v->ev_gather[v->gpar], v->st));
    v->gathered = v->running;
    v->gathered_stepped.assign(cnt, 0);
    for (int i = 0; i < cnt; ++i)
      v->gathered_stepped[i] = std::find(launched.begin(), launched.end(), v->running[i]) !=
                               launched.end();
    v->gather_pending = true;
    v->gpar ^= 1;
  }
  if (running) *running = (int)v->running.size();
  if (queued) *queued = (int)v->queue.size();
  return CLAW_OK;
}

claw_status claw_server_poll(claw_server* v, uint64_t ticket, void* q_host_out,
                             claw_req_info* info) {
  if (!v) return sfail(nullptr, "null server");
  auto it = v->reqs.find(ticket);
  if (it == v->reqs.end()) return sfail(v, "unknown ticket");
  Req& r = it->second;
  if (info) {
    info->status = r.status;
    info->steps = r.steps;
    info->t = r.t_reached;
    info->t_submit = r.t_submit;
    info->t_admit = r.t_admit;
    info->t_done = r.t_done;
  }
  if (r.status == CLAW_EBUSY) return CLAW_EBUSY;
  if (q_host_out && !r.result.empty()) std::memcpy(q_host_out, r.result.data(), r.result.size());
  const int st = r.status;
  v->reqs.erase(it);
  return st;
}

claw_status claw_server_take_done(claw_server* v, uint64_t* tickets, int cap, int* n) {
  if (!v || !n || cap < 0 || (cap > 0 && !tickets)) return sfail(v, "bad argument");
  int k = 0;
  while (k < cap && !v->completed.empty()) {
    tickets[k++] = v->completed.front();
    v->completed.pop_front();
  }
  *n = k;
  return CLAW_OK;
}

claw_status claw_server_schedule(claw_server* v, int policy, int64_t min_cells) {
  if (!v) return sfail(nullptr, "null server");
  if (policy != CLAW_SCHED_ALL && policy != CLAW_SCHED_SRW) return sfail(v, "unknown policy");
  if (policy == CLAW_SCHED_SRW && min_cells < 1) return sfail(v, "min_cells must be positive");
  v->sched = policy;
  if (policy == CLAW_SCHED_SRW) v->sched_cells = min_cells;
  return CLAW_OK;
}

claw_status claw_server_tune(claw_server* v, int mode, int* bw, int* h) {
  if (!v) return sfail(nullptr, "null server");
  const bool tunable = !v->faces && v->nd <= 2;
  if (tunable) {
    int nbw = v->bw, nh = v->h;
    if (mode == 0) {
      if (v->running.empty()) return sfail(v, "no running requests to tune on");
      std::vector<Member> hm;
      for (uint64_t t : v->running) hm.push_back(v->reqs[t].mem);
      VCK(cudaStreamSynchronize(v->st));
      VCK(tune_members(v->ks, v->nd, v->m, hm, v->consts.data(), v->st, nbw, nh));
    } else {
      if (!bw || !h) return sfail(v, "bad tile shape");
      const int want_bw = (v->m.scheme == CLAW_CLASSIC && v->nd == 1) ? v->bw : *bw;
      if (const char* why = bad_shape(v->ks, v->m, v->nd, want_bw, *h))
        return sfail(v, why);
      nbw = want_bw;
      nh = *h;
    }
    v->bw = nbw;
    v->h = nh;
    // running requests take the new shape from their next attempt on
    for (uint64_t t : v->running) {
      Req& r = v->reqs[t];
      r.mem.ntiles = tiles_of(v->m.scheme, v->nd, v->prec, v->ks.MA, r.mem.nx, r.mem.ny, v->bw,
                              v->h);
    }
    v->sel.clear();
    v->dirty = true;
  }
  if (bw) *bw = v->bw;
  if (h) *h = v->h;
  return CLAW_OK;
}

claw_status claw_server_destroy(claw_server* v) {
  if (!v) return CLAW_OK;
  if (v->st) cudaStreamSynchronize(v->st);
  for (auto& kv : v->reqs)
    if (kv.second.dblock) cudaFreeAsync(kv.second.dblock, v->st);
  if (v->d_mem) cudaFreeAsync(v->d_mem, v->st);
  if (v->d_tiles) cudaFreeAsync(v->d_tiles, v->st);
  if (v->d_stiles) cudaFreeAsync(v->d_stiles, v->st);
  if (v->d_tile0) cudaFreeAsync(v->d_tile0, v->st);
  if (v->d_smem) cudaFreeAsync(v->d_smem, v->st);
  if (v->d_gather) cudaFree(v->d_gather);
  if (v->h_gather) cudaFreeHost(v->h_gather);
  if (v->st) cudaStreamSynchronize(v->st);
  if (v->cst) cudaStreamSynchronize(v->cst);
  for (int k = 0; k < 2; ++k)
    if (v->ev_gather[k]) cudaEventDestroy(v->ev_gather[k]);
  if (v->ev_copy) cudaEventDestroy(v->ev_copy);
  if (v->ev_stage) cudaEventDestroy(v->ev_stage);
  if (v->stage) cudaFreeHost(v->stage);
  if (v->cst) cudaStreamDestroy(v->cst);
  if (v->st) cudaStreamDestroy(v->st);
  delete v;
  return CLAW_OK;
}

const char* claw_last_error(const void* handle) {
  (void)handle;
  return g_err.c_str();
}

const char* claw_version(void) { return kVersion; }

}  // extern "C"
