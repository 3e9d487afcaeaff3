// k_advection.cu -- fused kernels instantiated for the advection Riemann solver.
#include "launch.cuh"

namespace claw {

KernelSet claw_kernels_advection(int nd, int prec) {
  if (nd == 1 && prec == 0) return make_set<RpAdvection, 1, double>(true);
  if (nd == 1 && prec == 1) return make_set<RpAdvection, 1, float>(true);
  if (nd == 2 && prec == 0) return make_set<RpAdvection, 2, double>(true);
  if (nd == 2 && prec == 1) return make_set<RpAdvection, 2, float>(true);
  if (nd == 3 && prec == 0) return make_set<RpAdvection, 3, double>(false);
  if (nd == 3 && prec == 1) return make_set<RpAdvection, 3, float>(false);
  return KernelSet{};
}

}  // namespace claw
