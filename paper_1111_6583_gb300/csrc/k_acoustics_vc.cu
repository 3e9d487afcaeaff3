// k_acoustics_vc.cu -- fused kernels instantiated for acoustics in a varying
// medium.
#include "launch.cuh"

namespace claw {

KernelSet claw_kernels_acoustics_vc(int nd, int prec) {
  if (nd == 1 && prec == 0) return make_set<RpAcousticsVC, 1, double>(false);
  if (nd == 1 && prec == 1) return make_set<RpAcousticsVC, 1, float>(false);
  if (nd == 2 && prec == 0) return make_set<RpAcousticsVC, 2, double>(false);
  if (nd == 2 && prec == 1) return make_set<RpAcousticsVC, 2, float>(false);
  return KernelSet{};
}

}  // namespace claw
