// Constitutive kernels (x pass, commit, material point) in double, rate-solve variant NP = 10.
#include "kernels_impl.cuh"
namespace rve {
RVE_INSTANTIATE_X(double, 10)
}  // namespace rve
