// Common device types for the RVE solver kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rve {

template <typename T> struct C2t;
template <> struct C2t<float> { using type = float2; };
template <> struct C2t<double> { using type = double2; };
template <typename T> using C2 = typename C2t<T>::type;

template <typename T>
__device__ __forceinline__ C2<T> mk(T x, T y) { C2<T> r; r.x = x; r.y = y; return r; }
template <typename T>
__device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ C2<T> cmulc(C2<T> a, C2<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T>
__device__ __forceinline__ C2<T> cscale(C2<T> a, T s) { return mk<T>(a.x * s, a.y * s); }

// Threads per line in the first step of the two-step register transform of a line length
// n (n = N1 N2: 64 = 8 * 8, 96 = 8 * 12, 128 = 8 * 16, 160 = 10 * 16, 256 = 16 * 16; the
// PencilSplit table of fft_reg.cuh), 0 where n has no such split (those lengths run the
// Stockham kernels).
__host__ __device__ constexpr int pencil_n1(int n) {
  return (n == 64 || n == 96 || n == 128) ? 8 : (n == 160 ? 10 : (n == 256 ? 16 : 0));
}
// Largest kx chunk (HC) the two-step transforms of the y and z passes take: a CTA holds at
// most 384 threads, N1 for each of the chunk's 6 HC lines.
__host__ __device__ constexpr int pencil_max_hc(int n) { return pencil_n1(n) > 0 ? 384 / (6 * pencil_n1(n)) : 0; }

// One FFT length factored into radix stages (radices 2, 3, 4, 5).
struct FftDim {
  int n;
  int nst;
  int radix[12];
};

// Material constants on the device (Sec. 3, Sec. 4), plus the reference medium.
template <typename T>
struct MatDev {
  T C11, C12, C13, C33, C44, C66;
  T r0[16];
  T K, n, Kt, nt;
  T Q_s, Q_b, b_s, b_b;
  T h_diag, h_off;
  T c, d;
  T Kc, fm, eta;
  int n_int, nt_int;  // > 0 when n (nt) is that small integer: powers by multiplication
  T lam0, mu0;        // isotropic reference medium C0
  // starting point of the regularised-rate root (see reg_rate in constitutive.cuh)
  T inv_n, inv_nt;    // 1/n, 1/nt
  T sm, smt;          // smooth-min exponents: 1 / log2(1/u1), u1^n + u1 = 1
  T lg_K, lg_Kt;      // log2 K, log2 Kt
  T lg_eta;           // log2 eta (eta > 0)
  // Hooke's law scaled by the slip systems' Schmid factor 1/sqrt6 (shear rows with their
  // factor 2): the stage's resolved stresses come from C_s : e directly
  T C11s, C12s, C13s, C33s, C44s2, C66s2;
};

// Mixed-load controller data (always double).
struct LoadDev {
  double Minv[36];    // Mandel inverse of C0 restricted to the free components (zero elsewhere)
  double Sigma_m[6];  // target mean stress, Mandel
  int free_mask[6];   // 1 = stress-controlled
  int any_free;
  double s_ref;       // floor of the mean-stress norm in the relative errors (0: none)
};

// Per-iteration device record, written by the last CTA of each reduction.
struct IterStatus {
  double E[2][6];       // E^(i) in slot i%2 (tensor components)
  double sig_mean[6];   // <sigma>^(i)
  double cF;            // stress-constraint error
  double res_sum;       // sum_xi w |kappa . sigma_hat|^2
  double e_eq;          // equilibrium error
  double eff[4];        // commit: <sigma_eq>, <f_beta>, <v^s>, unused
  int nan_flag;
  int done;             // 0 iterating; 1 converged; 2 NaN/Inf; 3 iteration cap reached
  int done_it;          // iteration at which `done` was set
  int it_dev;           // device-driven iteration index (graph mode: advanced by the residual kernel)
  int guard;            // executions of the graph loop body (graph mode)
  int pad;
};

// Convergence rule evaluated on the device after each iteration's residual.
struct ConvDev {
  double tol;
  int fixed_iters;  // > 0: stop after exactly this many iterations
  int max_iter;
  double* hist;     // 2 * max_iter: (e_eq, c_F) of every iteration of the increment
  double s_ref;     // floor of the mean-stress norm in the relative errors (0: none)
};

constexpr int kNumRed = 9;  // reduction slots per CTA

// Regularised-rate root table (constitutive.cuh, reg_rate_tab): log2 u*(beta) as kRootIv
// linear pieces over log2 beta in [-kRootSpan, kRootSpan] (nodes every 1/kRootPerUnit,
// one at 0).  Interval i holds (a_i, b_i) with log2 u* = a_i + b_i t on it, in the
// absolute coordinate t = (log2 beta + kRootSpan) kRootPerUnit - 1/2.
constexpr int kRootIv = 2048;
constexpr double kRootSpan = 16.0;
constexpr double kRootPerUnit = kRootIv / (2.0 * kRootSpan);
constexpr int kRootTabLen = 2 * kRootIv;  // values per table
constexpr int kRootTabs = 2 * kRootTabLen;  // slip systems' table, then the twin exponent's

// Template value of the x pass's linear-law mode (the adjoint solve): s = B eps - g per voxel.
constexpr int kLinearLaw = 1;

// RK4 substeps whose start states the constitutive reverse pass (adjoint.cuh) keeps.
constexpr int kMaxSubVjp = 16;

}  // namespace rve
