// Constitutive kernels (x pass, commit, material point) in float, rate-solve variant NP = 0.
#include "kernels_impl.cuh"
namespace rve {
RVE_INSTANTIATE_X(float, 0)
}  // namespace rve
