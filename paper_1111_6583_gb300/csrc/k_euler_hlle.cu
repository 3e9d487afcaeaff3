// k_euler_hlle.cu -- fused kernels instantiated for the euler_hlle Riemann solver.
#include "launch.cuh"

namespace claw {

KernelSet claw_kernels_euler_hlle(int nd, int prec) {
  if (nd == 1 && prec == 0) return make_set<RpEulerHLLE, 1, double>(true);
  if (nd == 1 && prec == 1) return make_set<RpEulerHLLE, 1, float>(true);
  if (nd == 2 && prec == 0) return make_set<RpEulerHLLE, 2, double>(true);
  if (nd == 2 && prec == 1) return make_set<RpEulerHLLE, 2, float>(true);
  return KernelSet{};
}

}  // namespace claw
