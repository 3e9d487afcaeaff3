// k_euler_tracer.cu -- fused kernels instantiated for the Euler Roe solver
// with a passive tracer.
#include "launch.cuh"

namespace claw {

KernelSet claw_kernels_euler_tracer(int nd, int prec) {
  if (nd == 1 && prec == 0) return make_set<RpEulerTracer, 1, double>(true);
  if (nd == 1 && prec == 1) return make_set<RpEulerTracer, 1, float>(true);
  if (nd == 2 && prec == 0) return make_set<RpEulerTracer, 2, double>(true);
  if (nd == 2 && prec == 1) return make_set<RpEulerTracer, 2, float>(true);
  return KernelSet{};
}

}  // namespace claw
