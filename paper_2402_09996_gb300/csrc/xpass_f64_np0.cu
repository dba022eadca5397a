// Constitutive kernels (x pass, commit, material point) in double, rate-solve variant NP = 0.
#include "kernels_impl.cuh"
namespace rve {
RVE_INSTANTIATE_X(double, 0)
}  // namespace rve
