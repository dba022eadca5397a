// Constitutive kernels (x pass, commit, material point) in double, rate-solve variant NP = -1
// (eta > 0, real exponents).
#include "kernels_impl.cuh"
namespace rve {
RVE_INSTANTIATE_X(double, -1)
}  // namespace rve
