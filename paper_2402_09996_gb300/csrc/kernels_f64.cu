// double instantiation of the solver kernels and their launch wrappers.
#include "kernels_impl.cuh"
namespace rve {
RVE_INSTANTIATE(double)
}  // namespace rve
