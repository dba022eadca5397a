// Definitions of the launch wrappers, explicitly instantiated by kernels_f32.cu /
// kernels_f64.cu (FFT passes and helpers) and by xpass_<precision>_np<NP>.cu (the
// constitutive kernels, one rate-solve variant per translation unit).
#pragma once

#include "adjoint.cuh"
#include "launch.h"
#include "solver_kernels.cuh"

namespace rve {

// Opt in to the dynamic shared memory a launch needs (static shared memory counts
// towards the default 48 KB limit too, so any sizeable request sets the attribute).
template <typename T>
static cudaError_t set_smem(const void* fn, size_t smem) {
  if (smem <= 16 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T, int NP>
cudaError_t launch_xpass_np(const XArgs<T>& a, bool commit, int grid, size_t smem, cudaStream_t s) {
  if (commit) {
    cudaError_t e = set_smem<T>((const void*)k_xpass<T, true, NP>, smem);
    if (e != cudaSuccess) return e;
    k_xpass<T, true, NP><<<grid, kXThreads, smem, s>>>(a);
  } else {
    cudaError_t e = set_smem<T>((const void*)k_xpass<T, false, NP>, smem);
    if (e != cudaSuccess) return e;
    k_xpass<T, false, NP><<<grid, kXThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T, int NP>
cudaError_t launch_xpass_group_np(const XGroup<T>& g, bool commit, int grid, size_t smem, cudaStream_t s) {
  if (commit) {
    cudaError_t e = set_smem<T>((const void*)k_xpass_group<T, true, NP>, smem);
    if (e != cudaSuccess) return e;
    k_xpass_group<T, true, NP><<<grid, kXThreads, smem, s>>>(g);
  } else {
    cudaError_t e = set_smem<T>((const void*)k_xpass_group<T, false, NP>, smem);
    if (e != cudaSuccess) return e;
    k_xpass_group<T, false, NP><<<grid, kXThreads, smem, s>>>(g);
  }
  return cudaGetLastError();
}

template <typename T, int NP>
cudaError_t launch_material_point_np(const MatDev<T>& M, long long nvox, const T* R, const T* eps_n, const T* eps,
                                     T* state, T* sigma, T dt, int nsub, const T* root_tab, cudaStream_t s) {
  if (nvox <= 0) return cudaSuccess;
  const int thr = 128;
  const long long grid = (nvox + thr - 1) / thr;
  const size_t smem = (size_t)(kRootTabs) * sizeof(T);
  cudaError_t e = set_smem<T>((const void*)k_material_point<T, NP>, smem);
  if (e != cudaSuccess) return e;
  k_material_point<T, NP><<<(unsigned)grid, thr, smem, s>>>(M, nvox, R, eps_n, eps, state, sigma, dt, nsub,
                                                            root_tab);
  return cudaGetLastError();
}

template <typename T, int NP>
cudaError_t launch_material_point_vjp_np(const MatDev<T>& M, long long nvox, const T* R, const T* eps_n, const T* eps,
                                         const T* state, T dt, int nsub, const T* sigma_b, T* state_b, T* eps_b,
                                         T* eps_n_b, T* R_b, T* param_b, const T* root_tab, cudaStream_t s) {
  if (nvox <= 0) return cudaSuccess;
  const int thr = 64;
  const long long grid = (nvox + thr - 1) / thr;
  const size_t smem = (size_t)kRootTabs * sizeof(T);
  cudaError_t e = set_smem<T>((const void*)k_material_point_vjp<T, NP>, smem);
  if (e != cudaSuccess) return e;
  k_material_point_vjp<T, NP><<<(unsigned)grid, thr, smem, s>>>(M, nvox, R, eps_n, eps, state, dt, nsub, sigma_b,
                                                                state_b, eps_b, eps_n_b, R_b, param_b, root_tab);
  return cudaGetLastError();
}

template <typename T, int NP>
cudaError_t launch_adj_tangent_np(const MatDev<T>& M, long long nvox, const T* R, const T* eps_n, const T* eps,
                                  const T* state, T dt, int nsub, const double* sd, T* state_b, T* J, T* eps_b,
                                  T* eps_n_b, T* R_b, T* param_b, const T* root_tab, cudaStream_t s) {
  if (nvox <= 0) return cudaSuccess;
  const int thr = 64;
  const long long grid = (nvox + thr - 1) / thr;
  const size_t smem = (size_t)kRootTabs * sizeof(T);
  cudaError_t e = set_smem<T>((const void*)k_adj_tangent<T, NP>, smem);
  if (e != cudaSuccess) return e;
  k_adj_tangent<T, NP><<<(unsigned)grid, thr, smem, s>>>(M, nvox, R, eps_n, eps, state, dt, nsub, (T)sd[0], (T)sd[1],
                                                         (T)sd[2], (T)sd[3], (T)sd[4], (T)sd[5], state_b, J, eps_b,
                                                         eps_n_b, R_b, param_b, root_tab);
  return cudaGetLastError();
}

// the linear-law x pass alone (no material-point kernels)
#define RVE_INSTANTIATE_XLIN(T) \
  template cudaError_t launch_xpass_np<T, kLinearLaw>(const XArgs<T>&, bool, int, size_t, cudaStream_t);

#define RVE_INSTANTIATE_X(T, NP)                                                                                \
  template cudaError_t launch_xpass_np<T, NP>(const XArgs<T>&, bool, int, size_t, cudaStream_t);              \
  template cudaError_t launch_xpass_group_np<T, NP>(const XGroup<T>&, bool, int, size_t, cudaStream_t);       \
  template cudaError_t launch_material_point_np<T, NP>(const MatDev<T>&, long long, const T*, const T*, const T*, \
                                                       T*, T*, T, int, const T*, cudaStream_t);              \
  template cudaError_t launch_material_point_vjp_np<T, NP>(const MatDev<T>&, long long, const T*, const T*,      \
                                                           const T*, const T*, T, int, const T*, T*, T*, T*, T*, \
                                                           T*, const T*, cudaStream_t);                            \
  template cudaError_t launch_adj_tangent_np<T, NP>(const MatDev<T>&, long long, const T*, const T*, const T*,    \
                                                    const T*, T, int, const double*, T*, T*, T*, T*, T*, T*,       \
                                                    const T*, cudaStream_t);

// Threads of a pencil-pass CTA: N1 per line of the chunk (NC components of HC columns),
// rounded up to whole warps.
inline int pencil_threads(int n, int HC, int NC = 6) { return (pencil_n1(n) * NC * HC + 31) / 32 * 32; }
// The pencil kernels serve the component-interleaved passes whose length has a split and
// whose chunk fits one CTA.
inline bool pencil_ok(int n, int HC) { return HC <= pencil_max_hc(n); }

template <typename T, int SIGN, int N1, int N2, int NC>
static cudaError_t launch_line_pencil(const LineArgs<T>& a, dim3 grid, cudaStream_t s) {
  constexpr int N = N1 * N2;
  const size_t smem = ((size_t)N + (size_t)NC * a.HC * (N + 1)) * sizeof(C2<T>);
  cudaError_t e = set_smem<T>((const void*)k_line_pencil<T, SIGN, N1, N2, NC>, smem);
  if (e != cudaSuccess) return e;
  k_line_pencil<T, SIGN, N1, N2, NC><<<grid, pencil_threads(N, a.HC, NC), smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N, int NC>
static cudaError_t launch_line_pencil_n(const LineArgs<T>& a, int sign, dim3 grid, cudaStream_t s) {
  constexpr int N1 = PencilSplit<N>::N1, N2 = PencilSplit<N>::N2;
  return sign < 0 ? launch_line_pencil<T, -1, N1, N2, NC>(a, grid, s)
                  : launch_line_pencil<T, 1, N1, N2, NC>(a, grid, s);
}

template <typename T, int NC>
static cudaError_t launch_line_pencil_any(const LineArgs<T>& a, int sign, dim3 grid, cudaStream_t s) {
  switch (a.d.n) {
    case 64: return launch_line_pencil_n<T, 64, NC>(a, sign, grid, s);
    case 96: return launch_line_pencil_n<T, 96, NC>(a, sign, grid, s);
    case 128: return launch_line_pencil_n<T, 128, NC>(a, sign, grid, s);
    case 160: return launch_line_pencil_n<T, 160, NC>(a, sign, grid, s);
    default: return launch_line_pencil_n<T, 256, NC>(a, sign, grid, s);
  }
}

// The register two-step kernel serves a line length with a split when the chunk's lines fit
// one CTA: the solver's component-interleaved spectra (NC = hstride = 6) and the stand-alone
// transforms' component-major spectra (NC = hstride = 1).
template <typename T>
cudaError_t launch_line(const LineArgs<T>& a, int sign, dim3 grid, size_t smem, cudaStream_t s) {
  if (a.NC == 6 && a.hstride == 6 && pencil_ok(a.d.n, a.HC)) return launch_line_pencil_any<T, 6>(a, sign, grid, s);
  if (a.NC == 1 && a.hstride == 1 && pencil_n1(a.d.n) > 0 && pencil_n1(a.d.n) * a.HC <= kPencilThreads)
    return launch_line_pencil_any<T, 1>(a, sign, grid, s);
  if (sign < 0) {
    cudaError_t e = set_smem<T>((const void*)k_line<T, -1>, smem);
    if (e != cudaSuccess) return e;
    k_line<T, -1><<<grid, kLineThreads, smem, s>>>(a);
  } else {
    cudaError_t e = set_smem<T>((const void*)k_line<T, +1>, smem);
    if (e != cudaSuccess) return e;
    k_line<T, +1><<<grid, kLineThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T, int N1, int N2>
static cudaError_t launch_zgreen_pencil(const ZArgs<T>& a, dim3 grid, cudaStream_t s) {
  constexpr int N = N1 * N2;
  const size_t smem = ((size_t)N + (size_t)6 * a.HC * (N + 1)) * sizeof(C2<T>) + (size_t)a.HC * N * sizeof(double);
  cudaError_t e = set_smem<T>((const void*)k_zgreen<T, N1, N2>, smem);
  if (e != cudaSuccess) return e;
  k_zgreen<T, N1, N2><<<grid, pencil_threads(N, a.HC), smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zgreen(const ZArgs<T>& a, dim3 grid, size_t smem, cudaStream_t s) {
  if (pencil_ok(a.nz, a.HC)) {
    switch (a.nz) {
      case 64: return launch_zgreen_pencil<T, PencilSplit<64>::N1, PencilSplit<64>::N2>(a, grid, s);
      case 96: return launch_zgreen_pencil<T, PencilSplit<96>::N1, PencilSplit<96>::N2>(a, grid, s);
      case 128: return launch_zgreen_pencil<T, PencilSplit<128>::N1, PencilSplit<128>::N2>(a, grid, s);
      case 160: return launch_zgreen_pencil<T, PencilSplit<160>::N1, PencilSplit<160>::N2>(a, grid, s);
      default: return launch_zgreen_pencil<T, PencilSplit<256>::N1, PencilSplit<256>::N2>(a, grid, s);
    }
  }
  cudaError_t e = set_smem<T>((const void*)k_zgreen<T, 0, 0>, smem);
  if (e != cudaSuccess) return e;
  k_zgreen<T, 0, 0><<<grid, kZThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_line_group(const LineGroup<T>& g, int sign, int grid, size_t smem, cudaStream_t s) {
  if (sign < 0) {
    cudaError_t e = set_smem<T>((const void*)k_line_group<T, -1>, smem);
    if (e != cudaSuccess) return e;
    k_line_group<T, -1><<<grid, kPencilThreads, smem, s>>>(g);
  } else {
    cudaError_t e = set_smem<T>((const void*)k_line_group<T, +1>, smem);
    if (e != cudaSuccess) return e;
    k_line_group<T, +1><<<grid, kPencilThreads, smem, s>>>(g);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zgreen_group(const ZGroup<T>& g, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = set_smem<T>((const void*)k_zgreen_group<T>, smem);
  if (e != cudaSuccess) return e;
  k_zgreen_group<T><<<grid, kPencilThreads, smem, s>>>(g);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_group_guard(const GuardGroup& g, cudaGraphConditionalHandle cond, cudaStream_t s) {
  k_group_guard<T><<<1, 32, 0, s>>>(g, cond);
  return cudaGetLastError();
}

// Dynamic shared memory of a member's y / z pass CTA in the grouped kernels (the larger of
// the register-transform and Stockham layouts it may take).
template <typename T>
size_t line_group_smem(int n, int HC) {
  const size_t pencil = ((size_t)n + (size_t)6 * HC * (n + 1)) * sizeof(C2<T>);
  const size_t stock = ((size_t)n + (size_t)2 * 6 * HC * (n + 1)) * sizeof(C2<T>);
  return HC <= pencil_max_hc(n) ? pencil : stock;
}
template <typename T>
size_t zgreen_group_smem(int nz, int HC) {
  return line_group_smem<T>(nz, HC) + (size_t)HC * nz * sizeof(double);
}

template <typename T>
__global__ void k_shift_backup(C2<T>* spec, C2<T>* backup, long long NL, int H, double d0, double d1, double d2,
                               double d3, double d4, double d5, int restore) {
  // i = line * 6 + c; the kx = 0 entry of (line, c) is at line * H * 6 + c
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6 * NL) return;
  const int c = (int)(i % 6);
  C2<T>* p = spec + (size_t)(i / 6) * H * 6 + c;
  if (restore) {
    *p = backup[i];
    return;
  }
  backup[i] = *p;
  const double d = c == 0 ? d0 : c == 1 ? d1 : c == 2 ? d2 : c == 3 ? d3 : c == 4 ? d4 : d5;
  p->x = (T)((double)p->x + d);
}

template <typename T>
cudaError_t launch_shift(C2<T>* spec, C2<T>* backup, long long NL, int H, const double* dE, bool restore,
                         cudaStream_t s) {
  const long long n = 6 * NL;
  const int thr = 256;
  const long long grid = (n + thr - 1) / thr;
  k_shift_backup<T><<<(unsigned)grid, thr, 0, s>>>(spec, backup, NL, H, dE[0], dE[1], dE[2], dE[3], dE[4], dE[5],
                                                   restore ? 1 : 0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_xfft(const XFftArgs<T>& a, int sign, dim3 grid, size_t smem, cudaStream_t s) {
  if (sign < 0) {
    cudaError_t e = set_smem<T>((const void*)k_xfft<T, -1>, smem);
    if (e != cudaSuccess) return e;
    k_xfft<T, -1><<<grid, kXThreads, smem, s>>>(a);
  } else {
    cudaError_t e = set_smem<T>((const void*)k_xfft<T, +1>, smem);
    if (e != cudaSuccess) return e;
    k_xfft<T, +1><<<grid, kXThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_loop_guard(IterStatus* st, int limit, cudaGraphConditionalHandle cond, cudaStream_t s) {
  k_loop_guard<T><<<1, 32, 0, s>>>(st, limit, cond);
  return cudaGetLastError();
}

// dst = scale * src in double (scale 1: an exact widening copy)
template <typename T>
__global__ void k_to_double(const T* __restrict__ src, double* __restrict__ dst, long long n, double scale) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)src[i] * scale;
}

template <typename T>
cudaError_t launch_to_double(const T* src, double* dst, long long n, cudaStream_t s, double scale) {
  if (n <= 0) return cudaSuccess;
  const int thr = 256;
  k_to_double<T><<<(unsigned)((n + thr - 1) / thr), thr, 0, s>>>(src, dst, n, scale);
  return cudaGetLastError();
}

// double -> float (round to nearest)
template <typename T>
__global__ void k_to_float(const double* __restrict__ src, float* __restrict__ dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

template <typename T>
cudaError_t launch_to_float(const double* src, float* dst, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int thr = 256;
  k_to_float<T><<<(unsigned)((n + thr - 1) / thr), thr, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_von_mises(const T* __restrict__ sig, double* __restrict__ dst, long long nvox) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvox) return;
  T s[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) s[c] = sig[c * (size_t)nvox + i];
  dst[i] = (double)von_mises6<T>(s);
}

template <typename T>
cudaError_t launch_von_mises(const T* sig6, double* dst, long long nvox, cudaStream_t s) {
  if (nvox <= 0) return cudaSuccess;
  const int thr = 256;
  k_von_mises<T><<<(unsigned)((nvox + thr - 1) / thr), thr, 0, s>>>(sig6, dst, nvox);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- adjoint helpers ----
template <typename T>
__global__ void k_adj_gather_R(const uint32_t* __restrict__ grain, const T* __restrict__ Rg, T* __restrict__ Rvox,
                               long long nvox) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvox) return;
  const uint32_t g = grain[i];
  for (int k = 0; k < 9; ++k) Rvox[(size_t)i * 9 + k] = Rg[(size_t)g * 9 + k];
}

// out[c * nvox + i] = v[c] for all voxels (a uniform 6-vector field)
template <typename T>
__global__ void k_adj_fill6(T* out, double v0, double v1, double v2, double v3, double v4, double v5, long long nvox) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvox) return;
  const double v[6] = {v0, v1, v2, v3, v4, v5};
  for (int c = 0; c < 6; ++c) out[c * (size_t)nvox + i] = (T)v[c];
}

// Mandel-free pairing weights of the six components: the double contraction a : b of two
// symmetric tensors in (11 22 33 23 13 12) storage is sum_c w_c a_c b_c, w = (1 1 1 2 2 2).
__device__ __forceinline__ double adj_w(int c) { return c < 3 ? 1.0 : 2.0; }

// B(r, c) = J(c, r) w_c / w_r from the tangent rows J(k, .) = d sigma_k / d eps (the
// transposed tangent acting on tensors, in 6-component storage); g(r) = (e_a(r) + e_b(r)) / w_r.
template <typename T>
__global__ void k_adj_build(const T* __restrict__ Jrows, const T* __restrict__ ea, const T* __restrict__ eb,
                            T* __restrict__ B, T* __restrict__ g, long long nvox) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvox) return;
  const size_t n = (size_t)nvox;
  for (int r = 0; r < 6; ++r) {
    for (int c = 0; c < 6; ++c)
      B[(r * 6 + c) * n + i] = (T)((double)Jrows[(c * 6 + r) * n + i] * adj_w(c) / adj_w(r));
    g[r * n + i] = (T)(((double)ea[r * n + i] + (double)eb[r * n + i]) / adj_w(r));
  }
}

// sigma_b = -w mu (the stress adjoint of the equilibrium constraint)
template <typename T>
__global__ void k_adj_neg_w(const T* __restrict__ mu, T* __restrict__ sb, long long nvox) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvox) return;
  for (int c = 0; c < 6; ++c) sb[c * (size_t)nvox + i] = (T)(-adj_w(c) * (double)mu[c * (size_t)nvox + i]);
}

template <typename T>
__global__ void k_adj_from_double(const double* __restrict__ src, T* __restrict__ dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (T)src[i];
}

// dst = (double)(a + b)
template <typename T>
__global__ void k_adj_sum_to_double(const T* __restrict__ a, const T* __restrict__ b, double* __restrict__ dst,
                                    long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)a[i] + (double)b[i];
}

// Per-block partial sums of the tensor norm^2 of a 6-component field,
// sum_i f_c(i)^2 w_c (w = 1 1 1 2 2 2), in double and a fixed order: out[blockIdx.x].
template <typename T>
__global__ void k_adj_norm2(const T* __restrict__ f, double* __restrict__ out, long long nvox) {
  __shared__ double red[256 / 32];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double q = 0.0;
  if (i < nvox)
    for (int c = 0; c < 6; ++c) {
      const double x = (double)f[c * (size_t)nvox + i];
      q += adj_w(c) * x * x;
    }
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = q;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}

// Sum of A + B over 9 component rows (row k at k * nvox), in double: per-block partials
// out[blockIdx.x * 9 + k] (256 threads, fixed reduction order).
template <typename T>
__global__ void k_adj_param_sum(const T* __restrict__ A, const T* __restrict__ B, double* __restrict__ out,
                                long long nvox) {
  __shared__ double red[9][8];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    v[k] = i < nvox ? (double)A[k * (size_t)nvox + i] + (double)B[k * (size_t)nvox + i] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 9; ++k) red[k][threadIdx.x >> 5] = v[k];
  __syncthreads();
  if (threadIdx.x < 9) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[threadIdx.x][w];
    out[(size_t)blockIdx.x * 9 + threadIdx.x] = t;
  }
}

// Per-grain sums of A + B over 9 component rows: block g adds the voxels perm[goff[g] ..
// goff[g+1]) (one grain's voxels in increasing order) in a fixed order into out[g * 9 + k].
template <typename T>
__global__ void k_adj_grain_sum(const T* __restrict__ A, const T* __restrict__ B, const uint32_t* __restrict__ perm,
                                const int* __restrict__ goff, double* __restrict__ out, long long nvox) {
  __shared__ double red[9][8];
  const int g = blockIdx.x;
  double v[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) v[k] = 0.0;
  for (int j = goff[g] + threadIdx.x; j < goff[g + 1]; j += blockDim.x) {
    const size_t q = perm[j];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] += (double)A[k * (size_t)nvox + q] + (double)B[k * (size_t)nvox + q];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 9; ++k) red[k][threadIdx.x >> 5] = v[k];
  __syncthreads();
  if (threadIdx.x < 9) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[threadIdx.x][w];
    out[(size_t)g * 9 + threadIdx.x] = t;
  }
}

template <typename T>
cudaError_t launch_adj_sums(const T* pA, const T* pB, const T* rA, const T* rB, const uint32_t* perm, const int* goff,
                            int n_grains, long long nvox, double* param_part, double* grain_out, cudaStream_t s) {
  if (nvox <= 0) return cudaSuccess;
  const unsigned nb = (unsigned)((nvox + 255) / 256);
  k_adj_param_sum<T><<<nb, 256, 0, s>>>(pA, pB, param_part, nvox);
  if (n_grains > 0) k_adj_grain_sum<T><<<(unsigned)n_grains, 256, 0, s>>>(rA, rB, perm, goff, grain_out, nvox);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj(int which, long long n, cudaStream_t s, const void* p0, const void* p1, const void* p2,
                       void* q0, void* q1, const double* v) {
  const int thr = 256;
  const unsigned grid = (unsigned)((n + thr - 1) / thr);
  if (n <= 0) return cudaSuccess;
  switch (which) {
    case 0: k_adj_gather_R<T><<<grid, thr, 0, s>>>((const uint32_t*)p0, (const T*)p1, (T*)q0, n); break;
    case 1: k_adj_fill6<T><<<grid, thr, 0, s>>>((T*)q0, v[0], v[1], v[2], v[3], v[4], v[5], n); break;
    case 2: k_adj_build<T><<<grid, thr, 0, s>>>((const T*)p0, (const T*)p1, (const T*)p2, (T*)q0, (T*)q1, n); break;
    case 3: k_adj_neg_w<T><<<grid, thr, 0, s>>>((const T*)p0, (T*)q0, n); break;
    case 4: k_adj_from_double<T><<<grid, thr, 0, s>>>((const double*)p0, (T*)q0, n); break;
    case 5: k_adj_sum_to_double<T><<<grid, thr, 0, s>>>((const T*)p0, (const T*)p1, (double*)q0, n); break;
    case 6: k_adj_norm2<T><<<grid, thr, 0, s>>>((const T*)p0, (double*)q0, n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

#define RVE_INSTANTIATE(T)                                                                                         \
  template cudaError_t launch_line<T>(const LineArgs<T>&, int, dim3, size_t, cudaStream_t);                       \
  template cudaError_t launch_zgreen<T>(const ZArgs<T>&, dim3, size_t, cudaStream_t);                             \
  template cudaError_t launch_shift<T>(C2<T>*, C2<T>*, long long, int, const double*, bool, cudaStream_t);        \
  template cudaError_t launch_xfft<T>(const XFftArgs<T>&, int, dim3, size_t, cudaStream_t);                       \
  template cudaError_t launch_to_double<T>(const T*, double*, long long, cudaStream_t, double);                   \
  template cudaError_t launch_to_float<T>(const double*, float*, long long, cudaStream_t);                          \
  template cudaError_t launch_von_mises<T>(const T*, double*, long long, cudaStream_t);                          \
  template cudaError_t launch_loop_guard<T>(IterStatus*, int, cudaGraphConditionalHandle, cudaStream_t);           \
  template cudaError_t launch_adj<T>(int, long long, cudaStream_t, const void*, const void*, const void*, void*,   \
                                     void*, const double*);                                                        \
  template cudaError_t launch_adj_sums<T>(const T*, const T*, const T*, const T*, const uint32_t*, const int*, int, \
                                          long long, double*, double*, cudaStream_t);                              \
  template cudaError_t launch_line_group<T>(const LineGroup<T>&, int, int, size_t, cudaStream_t);                  \
  template cudaError_t launch_zgreen_group<T>(const ZGroup<T>&, int, size_t, cudaStream_t);                        \
  template cudaError_t launch_group_guard<T>(const GuardGroup&, cudaGraphConditionalHandle, cudaStream_t);         \
  template size_t line_group_smem<T>(int, int);                                                                    \
  template size_t zgreen_group_smem<T>(int, int);

}  // namespace rve
