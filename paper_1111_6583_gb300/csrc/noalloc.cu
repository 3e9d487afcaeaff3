// noalloc.cu -- a SharpClaw step that allocates no memory.
//
// Some callers cannot let a library call cudaMalloc: applications whose
// device memory is owned entirely by their own allocator or fixed arena (a
// framework's caching allocator, a solver embedded in a larger code that
// budgets every byte), and code paths where an allocation would synchronise
// the device or is not permitted.  claw_sharp_step_noalloc serves them: the
// caller passes the input and output states, and everything else the step
// needs -- the two intermediate SSP-RK3 stage states, the control block that
// collects the wave speeds, and the grid descriptors -- lives in one
// file-scope device array, kNoallocScratchBytes long, that every GPU which
// loads the library holds until the process exits.
//
// Set-up: the first call on each device (with that device current) looks up
// the array's device address with cudaGetSymbolAddress; make that first call
// before any stream capture.  All calls share the array and it keeps the
// last call's contents; the control block is rewritten (its accumulators
// zeroed) at the start of every call.  Calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "claw_common.cuh"
#include "kernels.h"

using namespace claw;

namespace {

constexpr size_t kNoallocScratchBytes = 8u << 20;  // 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (looked up once)
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// errors are reported through claw_last_error
claw_status nfail(const std::string& msg, cudaError_t e = cudaSuccess) {
  std::string m = msg;
  if (e != cudaSuccess) m += std::string(": ") + cudaGetErrorString(e);
  claw::set_last_error(m.c_str());
  return e != cudaSuccess ? CLAW_ECUDA : CLAW_EINVAL;
}

}  // namespace

extern "C" {

claw_status claw_sharp_step_noalloc(const claw_method* m, const claw_grid* g, const void* q_in,
                                    void* q_out, const void* aux, double dt, void* stream,
                                    double* cfl) {
  if (!m || !g || !q_in || !q_out) return nfail("null argument");
  // the checks of the handle API first (grid extents up to INT_MAX / 2,
  // num_eqn and num_aux against the solver, limiter, precision, boundaries...)
  if (const char* why = validate_grid(*g, *m)) return nfail(why);
  if (const char* why = validate_method(*m, g->ndim)) return nfail(why);
  // then what this step does not take
  if (m->scheme != CLAW_SHARPCLAW) return nfail("claw_sharp_step_noalloc needs scheme SharpClaw");
  if (g->ndim != 1 && g->ndim != 2) return nfail("ndim must be 1 or 2");
  if (m->weno_order != 5) return nfail("the allocation-free step takes WENO5 only");
  if (m->time_integrator != CLAW_SSP_RK3)
    return nfail("the allocation-free step takes the SSP-RK3 integrator only");
  if (m->capa_index != -1 || m->source != CLAW_SOURCE_NONE)
    return nfail("the allocation-free step takes no capacity or source term");
  if (!(dt > 0)) return nfail("dt must be positive");
  KernelSet ks = kernels_of(m->rp, g->ndim, m->prec);
  if (!ks.valid || ks.M != m->num_eqn || !ks.sharp)
    return nfail("unsupported solver/dimension/precision");
  if (m->num_aux != ks.MA) return nfail("num_aux does not match the Riemann solver");
  if (ks.MA > 0 && !aux) return nfail("this solver needs aux fields");
  if (q_in == q_out) return nfail("q_in and q_out must be different buffers");
  const int nx = (int)g->n[0], ny = g->ndim == 2 ? (int)g->n[1] : 1;
  // cell count first, so the byte count below cannot wrap
  if ((size_t)nx * (size_t)ny > kNoallocScratchBytes)
    return nfail("grid too large for the no-allocation step: more cells than the " +
                 std::to_string(kNoallocScratchBytes) + "-byte scratch array holds");

  // scratch layout: [stage 1 state][stage 2 state][control block][2 descriptors]
  const size_t es = m->prec == CLAW_FP64 ? 8 : 4;
  const size_t sb = al256((size_t)nx * ny * m->num_eqn * es);
  const size_t need = 2 * sb + al256(sizeof(DevCtl)) + 2 * al256(sizeof(Member));
  if (need > kNoallocScratchBytes)
    return nfail("grid too large for the no-allocation step: needs " + std::to_string(need) +
                 " bytes of scratch, the maximum is " + std::to_string(kNoallocScratchBytes));

  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return nfail("cudaGetSymbolAddress of the scratch array", e);
  unsigned char* p = (unsigned char*)base;
  void* q1 = p;
  void* q2 = p + sb;
  DevCtl* ctl = (DevCtl*)(p + 2 * sb);
  Member* mem = (Member*)(p + 2 * sb + al256(sizeof(DevCtl)));
  Member* mem_last = (Member*)((unsigned char*)mem + al256(sizeof(Member)));
  cudaStream_t st = (cudaStream_t)stream;

  // control block: forced step of size dt from t = 0; accumulators zeroed
  DevCtl c;
  std::memset(&c, 0, sizeof(c));
  c.dt = dt;
  c.t_end = INFINITY;
  c.dt_max = INFINITY;
  c.cfl_desired = 1.0;
  c.cfl_max = INFINITY;
  c.dx[0] = (g->upper[0] - g->lower[0]) / (double)nx;
  c.dx[1] = g->ndim == 2 ? (g->upper[1] - g->lower[1]) / (double)ny : 1.0;
  c.dx[2] = 1.0;
  for (int d = 0; d < 3; ++d) c.idx[d] = 1.0 / c.dx[d];
  c.max_steps = 0x7fffffffffffffffLL;
  c.nbuf = 3;
  c.accept_shift = 1;
  c.forced = 1;
  c.ndim = g->ndim;
  // stages 0 and 1: Q^n -> Q1 -> Q2 in scratch; stage 2 reads Q2, writes q_out
  Member h[2];
  std::memset(h, 0, sizeof(h));
  h[0].q[0] = (void*)q_in;
  h[0].q[1] = q1;
  h[0].q[2] = q2;
  h[0].aux = aux;
  h[0].nx = nx;
  h[0].ny = ny;
  h[0].ctl = ctl;
  h[1] = h[0];
  h[1].q[1] = q_out;
  const int ntiles =
      g->ndim == 1 ? sharp_tiles(nx, 1, kSharpTX1, 1) : sharp_tiles(nx, ny, kSharpTX2, kSharpTY2);
  h[0].ntiles = h[1].ntiles = ntiles;
  if ((e = cudaMemcpyAsync(ctl, &c, sizeof(DevCtl), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return nfail("control block upload", e);
  if ((e = cudaMemcpyAsync(mem, &h[0], sizeof(Member), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return nfail("descriptor upload", e);
  if ((e = cudaMemcpyAsync(mem_last, &h[1], sizeof(Member), cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return nfail("descriptor upload", e);

  // method constants on the host stack: the kernels take them by value
  alignas(16) unsigned char consts[sizeof(MConsts<double>)];
  {
    const std::vector<unsigned char> v = method_consts(*m);
    if (v.size() > sizeof(consts)) return nfail("method constants do not fit");
    std::memcpy(consts, v.data(), v.size());
  }
  for (int s = 0; s < 3; ++s) {
    LaunchArgs a{s < 2 ? mem : mem_last, nullptr, ntiles, consts, 0, 0, s, st};
    if ((e = ks.sharp(a)) != cudaSuccess) return nfail("stage launch", e);
  }
  DevCtl out;
  if ((e = cudaMemcpyAsync(&out, ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return nfail("control block read", e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return nfail("step", e);
  if (cfl) *cfl = out.nu_last;
  if (out.status != CLAW_OK) {
    claw::set_last_error("step produced non-finite values");
    return out.status;
  }
  return CLAW_OK;
}

}  // extern "C"
