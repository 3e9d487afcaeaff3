// k_elasticity.cu -- fused kernels instantiated for the elasticity Riemann solver.
#include "launch.cuh"

namespace claw {

KernelSet claw_kernels_elasticity(int nd, int prec) {
  if (nd == 1 && prec == 0) return make_set<RpElasticity, 1, double>(false);
  if (nd == 1 && prec == 1) return make_set<RpElasticity, 1, float>(false);
  if (nd == 2 && prec == 0) return make_set<RpElasticity, 2, double>(false);
  if (nd == 2 && prec == 1) return make_set<RpElasticity, 2, float>(false);
  return KernelSet{};
}

}  // namespace claw
