// Linear-law x pass in float (the adjoint solve: s = B eps - g per voxel).
#include "kernels_impl.cuh"
namespace rve {
RVE_INSTANTIATE_XLIN(float)
}  // namespace rve
