// k_euler_roe.cu -- fused kernels instantiated for the euler_roe Riemann solver.
#include "launch.cuh"

namespace claw {

KernelSet claw_kernels_euler_roe(int nd, int prec) {
  if (nd == 1 && prec == 0) return make_set<RpEulerRoe, 1, double>(true);
  if (nd == 1 && prec == 1) return make_set<RpEulerRoe, 1, float>(true);
  if (nd == 2 && prec == 0) return make_set<RpEulerRoe, 2, double>(true);
  if (nd == 2 && prec == 1) return make_set<RpEulerRoe, 2, float>(true);
  return KernelSet{};
}

}  // namespace claw
