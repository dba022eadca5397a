// Host launch wrappers for the solver kernels (one instantiation per precision).
#pragma once

#include <cuda_runtime.h>

#include "rve_common.cuh"

namespace rve {

template <typename T> struct XArgs;
template <typename T> struct LineArgs;
template <typename T> struct ZArgs;
template <typename T> struct XFftArgs;
template <typename T> struct XGroup;
template <typename T> struct LineGroup;
template <typename T> struct ZGroup;
struct GuardGroup;

// Rate-solve variants of the constitutive kernels (see constitutive.cuh): NP = 10 for
// n = nt = 10 and eta >= max(K, Kt) (the floored solve, root_floor, is exact there), NP = -1
// for eta > 0 otherwise (exponents >= 1), NP = 0 (generic per-system solve) for eta = 0.
inline int rate_variant(double eta, double K, double Kt, int n_int, int nt_int) {
  if (!(eta > 0.0)) return 0;
  return (n_int == 10 && nt_int == 10 && eta >= K && eta >= Kt) ? 10 : -1;
}

// Per-variant entry points (each instantiated in its own translation unit).
template <typename T, int NP>
cudaError_t launch_xpass_np(const XArgs<T>& a, bool commit, int grid, size_t smem, cudaStream_t s);
template <typename T, int NP>
cudaError_t launch_material_point_np(const MatDev<T>& M, long long nvox, const T* R, const T* eps_n, const T* eps,
                                     T* state, T* sigma, T dt, int nsub, const T* root_tab, cudaStream_t s);

template <typename T, int NP>
cudaError_t launch_material_point_vjp_np(const MatDev<T>& M, long long nvox, const T* R, const T* eps_n, const T* eps,
                                         const T* state, T dt, int nsub, const T* sigma_b, T* state_b, T* eps_b,
                                         T* eps_n_b, T* R_b, T* param_b, const T* root_tab, cudaStream_t s);

template <typename T, int NP>
cudaError_t launch_adj_tangent_np(const MatDev<T>& M, long long nvox, const T* R, const T* eps_n, const T* eps,
                                  const T* state, T dt, int nsub, const double* sd, T* state_b, T* J, T* eps_b,
                                  T* eps_n_b, T* R_b, T* param_b, const T* root_tab, cudaStream_t s);

// tangent rows and direct part of one increment's adjoint (adjoint.cuh, k_adj_tangent)
template <typename T>
cudaError_t launch_adj_tangent(const MatDev<T>& M, int np, long long nvox, const T* R, const T* eps_n, const T* eps,
                               const T* state, T dt, int nsub, const double* sd, T* state_b, T* J, T* eps_b,
                               T* eps_n_b, T* R_b, T* param_b, const T* root_tab, cudaStream_t s) {
  if (np == 10)
    return launch_adj_tangent_np<T, 10>(M, nvox, R, eps_n, eps, state, dt, nsub, sd, state_b, J, eps_b, eps_n_b, R_b,
                                        param_b, root_tab, s);
  if (np < 0)
    return launch_adj_tangent_np<T, -1>(M, nvox, R, eps_n, eps, state, dt, nsub, sd, state_b, J, eps_b, eps_n_b, R_b,
                                        param_b, root_tab, s);
  return launch_adj_tangent_np<T, 0>(M, nvox, R, eps_n, eps, state, dt, nsub, sd, state_b, J, eps_b, eps_n_b, R_b,
                                     param_b, root_tab, s);
}

template <typename T>
cudaError_t launch_material_point_vjp(const MatDev<T>& M, int np, long long nvox, const T* R, const T* eps_n,
                                      const T* eps, const T* state, T dt, int nsub, const T* sigma_b, T* state_b,
                                      T* eps_b, T* eps_n_b, T* R_b, T* param_b, const T* root_tab, cudaStream_t s) {
  if (np == 10)
    return launch_material_point_vjp_np<T, 10>(M, nvox, R, eps_n, eps, state, dt, nsub, sigma_b, state_b, eps_b,
                                               eps_n_b, R_b, param_b, root_tab, s);
  if (np < 0)
    return launch_material_point_vjp_np<T, -1>(M, nvox, R, eps_n, eps, state, dt, nsub, sigma_b, state_b, eps_b,
                                               eps_n_b, R_b, param_b, root_tab, s);
  return launch_material_point_vjp_np<T, 0>(M, nvox, R, eps_n, eps, state, dt, nsub, sigma_b, state_b, eps_b,
                                            eps_n_b, R_b, param_b, root_tab, s);
}

template <typename T>
cudaError_t launch_xpass(const XArgs<T>& a, int np, bool commit, int grid, size_t smem, cudaStream_t s) {
  if (np == 10) return launch_xpass_np<T, 10>(a, commit, grid, smem, s);
  if (np == kLinearLaw) return launch_xpass_np<T, kLinearLaw>(a, commit, grid, smem, s);
  if (np < 0) return launch_xpass_np<T, -1>(a, commit, grid, smem, s);
  return launch_xpass_np<T, 0>(a, commit, grid, smem, s);
}
template <typename T>
cudaError_t launch_material_point(const MatDev<T>& M, int np, long long nvox, const T* R, const T* eps_n, const T* eps,
                                  T* state, T* sigma, T dt, int nsub, const T* root_tab, cudaStream_t s) {
  if (np == 10) return launch_material_point_np<T, 10>(M, nvox, R, eps_n, eps, state, sigma, dt, nsub, root_tab, s);
  if (np < 0) return launch_material_point_np<T, -1>(M, nvox, R, eps_n, eps, state, sigma, dt, nsub, root_tab, s);
  return launch_material_point_np<T, 0>(M, nvox, R, eps_n, eps, state, sigma, dt, nsub, root_tab, s);
}

template <typename T>
cudaError_t launch_line(const LineArgs<T>& a, int sign, dim3 grid, size_t smem, cudaStream_t s);
// grouped passes (solver_kernels.cuh, k_*_group): one launch over several RVEs' grids; the
// grouped x pass per rate variant as launch_xpass
template <typename T, int NP>
cudaError_t launch_xpass_group_np(const XGroup<T>& g, bool commit, int grid, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_xpass_group(const XGroup<T>& g, int np, bool commit, int grid, size_t smem, cudaStream_t s) {
  if (np == 10) return launch_xpass_group_np<T, 10>(g, commit, grid, smem, s);
  if (np < 0) return launch_xpass_group_np<T, -1>(g, commit, grid, smem, s);
  return launch_xpass_group_np<T, 0>(g, commit, grid, smem, s);
}
template <typename T>
cudaError_t launch_line_group(const LineGroup<T>& g, int sign, int grid, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_zgreen_group(const ZGroup<T>& g, int grid, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_group_guard(const GuardGroup& g, cudaGraphConditionalHandle cond, cudaStream_t s);
template <typename T>
size_t line_group_smem(int n, int HC);
template <typename T>
size_t zgreen_group_smem(int nz, int HC);
template <typename T>
cudaError_t launch_zgreen(const ZArgs<T>& a, dim3 grid, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_shift(C2<T>* spec, C2<T>* backup, long long NL, int H, const double* dE, bool restore,
                         cudaStream_t s);
template <typename T>
cudaError_t launch_xfft(const XFftArgs<T>& a, int sign, dim3 grid, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_to_double(const T* src, double* dst, long long n, cudaStream_t s, double scale = 1.0);
template <typename T>
cudaError_t launch_to_float(const double* src, float* dst, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_von_mises(const T* sig6, double* dst, long long nvox, cudaStream_t s);
template <typename T>
cudaError_t launch_loop_guard(IterStatus* st, int limit, cudaGraphConditionalHandle cond, cudaStream_t s);
// adjoint gradient sums (kernels_impl.cuh): per-block partial sums of the 9 parameter rows
// pA + pB (param_part, 9 per block of 256 voxels) and per-grain sums of the 9 rotation rows
// rA + rB over the grain-sorted voxel list perm / goff (grain_out, 9 per grain)
template <typename T>
cudaError_t launch_adj_sums(const T* pA, const T* pB, const T* rA, const T* rB, const uint32_t* perm, const int* goff,
                            int n_grains, long long nvox, double* param_part, double* grain_out, cudaStream_t s);
// adjoint helpers (kernels_impl.cuh): 0 gather per-voxel R, 1 fill a uniform 6-vector field,
// 2 build B and g, 3 sigma_b = -w mu, 4 double -> T copy, 5 T + T -> double sum
template <typename T>
cudaError_t launch_adj(int which, long long n, cudaStream_t s, const void* p0, const void* p1, const void* p2,
                       void* q0, void* q1, const double* v);

int x_threads();
int line_threads();
int z_threads();

}  // namespace rve
