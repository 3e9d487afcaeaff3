// kernels.h -- host-side view of the per-solver kernel sets (no CUDA types
// beyond the runtime API).  Each k_<solver>.cu translation unit instantiates
// the fused kernels for its Riemann solver in FP64 and FP32 and returns their
// launchers through claw_kernels_<solver>().
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "clawgpu.h"

namespace claw {

struct Member;
struct Tile;
struct DevCtl;
struct StageOp;

struct LaunchArgs {
  const Member* members;   // device array
  const Tile* tiles;       // device array or nullptr (single member, tiles 0..n-1)
  int ntiles_total;        // work items of this launch
  const void* consts;      // host pointer to MConsts<R>
  int bw;                  // 2D classic: threads per block (strip width + 4)
  int h;                   // 2D classic: rows per block; 1D classic: how warps take
                           // work (kWork1dTiles, kWork1dUnits, else automatic)
  int stage;               // SharpClaw SSP-RK3 stage 0..2 (used when stage_op is null)
  cudaStream_t stream;
  int n3[3];               // 3D: cells per direction
  void* work3;             // 3D: per-face arrays (device)
  size_t work3_bytes;
  const StageOp* stage_op; // SharpClaw: explicit stage (host pointer) or null
  int sweep;               // 2D classic: 0 unsplit, 1 / 2 the x / y sweeps of a split step
  int nmembers;            // members of the table (1D classic runs their controllers after)
  int src_phase;           // source step: 0 Godunov (dt after an accepted step), 1 Strang
                           // pre (dt/2 of the attempt, slot cur -> qpre), 2 Strang post
                           // (dt/2 after an accepted step)
};

// stage tables of the SharpClaw time integrators
int stage_table(int integrator, const StageOp** ops);  // returns the number of stages

typedef cudaError_t (*launch_fn)(const LaunchArgs&);

struct KernelSet {
  int valid;
  int M, MW, MA;
  int has_char;            // characteristic projection available
  launch_fn classic;       // one attempt (1D or 2D by the member grid)
  launch_fn sharp;         // one SSP-RK3 stage
  launch_fn maxspeed;      // first-order interface speeds into ctl->smax
  launch_fn source;        // axisymmetric Euler source step (2D Euler systems)
  int max_bw;              // 2D classic: widest block whose static shared memory fits
  int sharp_shapes;        // 2D SharpClaw WENO5: bit i set when tile kSharpShapes2[i]
                           // fits in a block's shared memory
};

// tile geometry shared by the host (tile tables) and the kernels
constexpr int kClassic1dThreads = 128;
// cells per lane: FP64 2 (more warps for the small single grids the FP64
// form runs); FP32 8 for solvers without aux fields (two 16-byte loads per
// field: 2^26-cell acoustics 0.42 -> 0.28 ms) and 4 for solvers that read
// aux fields (the elasticity ensemble is faster with 4: 0.59 vs 0.76 ms)
constexpr int classic1d_K(int prec, int ma) { return prec == 0 ? 2 : (ma == 0 ? 8 : 4); }
// staged form: slots of the shared-memory ring per warp through which bulk
// asynchronous copies deliver the units (0: direct loads).  FP32 solvers of
// one or two fields without aux fields (the streaming-bound ones); FP64,
// bound by the FP64 pipe, and the heavier solvers, bound by instruction
// issue, keep the direct loads.
constexpr int classic1d_S(int prec, int m, int ma) {
  return prec == 1 && ma == 0 && m <= 2 ? 3 : 0;
}
// a warp writes the cells of its lanes 1..30 (lanes 0 and 31 hold its halo)
constexpr int classic1d_T(int prec, int ma) {
  return kClassic1dThreads / 32 * 30 * classic1d_K(prec, ma);
}
inline int classic1d_tiles(int nx, int prec, int ma) {
  return (nx + classic1d_T(prec, ma) - 1) / classic1d_T(prec, ma);
}
// 1D classic work modes (LaunchArgs::h): a warp takes a whole tile, or one
// unit of it; any other value: whole tiles when they fill every resident warp
constexpr int kWork1dTiles = 1, kWork1dUnits = 2;
constexpr int kSharpTX2 = 16, kSharpTY2 = 8;  // 2D SharpClaw tile (default)
constexpr int kSharpTX1 = 128;                // 1D SharpClaw tile
// shared memory one block may hold on the device (227 KB)
constexpr size_t kSmemPerBlock = 227 * 1024;
// 2D SharpClaw tiles (TX, TY) of the fifth-order WENO stage that the
// autotuner tries; the higher orders keep the default
constexpr int kSharpShapes2[4][2] = {{16, 8}, {32, 4}, {32, 8}, {16, 16}};
// the 2D SharpClaw tile that a launch shape (bw, h) names: one of
// kSharpShapes2, any other pair the default
inline void sharp2d_shape(int bw, int h, int& tx, int& ty) {
  tx = kSharpTX2;
  ty = kSharpTY2;
  for (const auto& sh : kSharpShapes2)
    if (sh[0] == bw && sh[1] == h) {
      tx = bw;
      ty = h;
    }
}
constexpr int kMaxspeedCells = 256;           // cells per max-speed block

// Tiles of the 2D classic kernel.  A block of BW threads owns a strip of
// TX = BW - 4 interior columns and a chunk of rows; the ny rows are spread
// evenly over nch = ceil(ny / H) chunks (no short last chunk).  Tile t is
// strip t % nsx, chunk t / nsx.  In a narrow last strip the warps that hold
// only columns past the second ghost column skip all work; its chunks keep
// the common height, since a tile's time is set by the rows each of its warps
// walks, not by the number of warps.
struct Classic2dLayout {
  int TX, nsx, nch;
};
__host__ __device__ inline Classic2dLayout classic2d_layout(int nx, int ny, int BW, int H) {
  Classic2dLayout L;
  L.TX = BW - 4;
  L.nsx = (nx + L.TX - 1) / L.TX;
  L.nch = (ny + H - 1) / H;
  return L;
}
__host__ __device__ inline int classic2d_tiles(int nx, int ny, int BW, int H) {
  const Classic2dLayout L = classic2d_layout(nx, ny, BW, H);
  return L.nsx * L.nch;
}
__host__ __device__ inline int sharp_tiles(int nx, int ny, int TX, int TY) {
  return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
}

// 3D update: cells per block (256 threads, four cells each); the update's
// blocks count the arrivals for the controller
constexpr int kUpdateCells3d = 1024;
inline int classic3d_update_blocks(long long cells) {
  return (int)((cells + kUpdateCells3d - 1) / kUpdateCells3d);
}

inline size_t classic3d_work_bytes(int nx, int ny, int nz, int M, int prec) {
  size_t faces = (size_t)(nx + 1) * ny * nz + (size_t)nx * (ny + 1) * nz + (size_t)nx * ny * (nz + 1);
  return faces * 3 * M * (prec == 0 ? 8 : 4);
}

KernelSet claw_kernels_advection(int nd, int prec);
KernelSet claw_kernels_acoustics(int nd, int prec);
KernelSet claw_kernels_sw(int nd, int prec);
KernelSet claw_kernels_euler_roe(int nd, int prec);
KernelSet claw_kernels_euler_hlle(int nd, int prec);
KernelSet claw_kernels_elasticity(int nd, int prec);
KernelSet claw_kernels_euler_tracer(int nd, int prec);
KernelSet claw_kernels_acoustics_vc(int nd, int prec);
// bytes of the per-face records of the per-face classic path
size_t faces_work_bytes(int nd, int nx, int ny, int m, int prec);

// generic kernels (k_common.cu)
cudaError_t launch_dt_init(DevCtl* ctls, int n, cudaStream_t st);
// after a source launch: record that every member's accepted steps have had
// their source step (members[k].ctl->src_mark = steps)
cudaError_t launch_source_mark(const Member* members, int n, cudaStream_t st);
// the CFL controller of every member that took part in the attempt (not done)
cudaError_t launch_controllers(const Member* members, int n, cudaStream_t st);
cudaError_t launch_set_t_end(DevCtl* ctls, int n, double t_end, long long max_steps_rel,
                             cudaStream_t st);
cudaError_t launch_force_dt(DevCtl* ctl, double dt, cudaStream_t st);
cudaError_t launch_count_active(const DevCtl* ctls, int n, int* out, cudaStream_t st);
cudaError_t launch_totals(const void* q, const void* kappa, int prec, long long ncell, int m,
                          double* partials, int nblocks, cudaStream_t st);
cudaError_t launch_reset_cur(DevCtl* ctl, cudaStream_t st);
cudaError_t launch_gather_ctl(const Member* members, int n, DevCtl* out, cudaStream_t st);
cudaError_t launch_set_dry(DevCtl* ctl, int dry, cudaStream_t st);
cudaError_t launch_set_dry_n(DevCtl* ctls, int n, int dry, cudaStream_t st);
constexpr int kTotalsThreads = 256;

// record the message that claw_last_error returns (api.cu)
void set_last_error(const char* msg);

// argument checks of the handle API (nullptr when valid, else the reason),
// the method constants MConsts<R> as bytes, and a solver's kernel set (api.cu)
const char* validate_method(const claw_method& m, int nd);
const char* validate_grid(const claw_grid& g, const claw_method& m);
std::vector<unsigned char> method_consts(const claw_method& m);
KernelSet kernels_of(int rp, int nd, int prec);

}  // namespace claw
