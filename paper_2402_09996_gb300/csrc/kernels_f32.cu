// float instantiation of the solver kernels and their launch wrappers.
#include "kernels_impl.cuh"
namespace rve {
RVE_INSTANTIATE(float)
int x_threads() { return kXThreads; }
int line_threads() { return kLineThreads; }
int z_threads() { return kZThreads; }
}  // namespace rve
