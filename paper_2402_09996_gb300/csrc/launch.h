// Host launch wrappers for the solver kernels (one instantiation per precision).
#pragma once

#include <cuda_runtime.h>

#include "rve_common.cuh"

namespace rve {

template <typename T> struct XArgs;
template <typename T> struct LineArgs;
template <typename T> struct ZArgs;
template <typename T> struct XFftArgs;

template <typename T>
cudaError_t launch_xpass(const XArgs<T>& a, bool commit, int grid, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_line(const LineArgs<T>& a, int sign, dim3 grid, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_zgreen(const ZArgs<T>& a, dim3 grid, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_shift(C2<T>* spec, C2<T>* backup, long long NL, int H, const double* dE, bool restore,
                         cudaStream_t s);
template <typename T>
cudaError_t launch_material_point(const MatDev<T>& M, long long nvox, const T* R, const T* eps_n, const T* eps,
                                  T* state, T* sigma, T dt, int nsub, cudaStream_t s);
template <typename T>
cudaError_t launch_xfft(const XFftArgs<T>& a, int sign, dim3 grid, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_to_double(const T* src, double* dst, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_von_mises(const T* sig6, double* dst, long long nvox, cudaStream_t s);

int x_threads();
int line_threads();
int z_threads();

}  // namespace rve
