// Per-voxel Meric-Cailletaud crystal plasticity (arXiv 2402.09996, Sec. 3 and 4).
//
// State (crystal frame): plastic strain eps_p (6 tensor components, order 11 22 33 23
// 13 12), accumulated slip v (12 slip systems then 4 twin systems; the twin volume
// fraction is f = sqrt(2) v), kinematic variables alpha of the 12 slip systems.
//
// Rates at strain eps (Sec. 3):
//   sigma   = C : (eps - eps_p)                                 (tetragonal C, c || z)
//   tau     = sigma : m,  m = (n x l + l x n)/2                 (Table 1 systems)
//   r       = r0 + Q sum_s' q_ss' (1 - exp(-b v_s'))            (q = h_diag / h_off)
//   slip:   a = |tau - c alpha| - r,  gdot = sign(tau - c alpha) rho,
//           rho = < (a - eta rho) / K >^n                       (Sec. 4, Eq. (regu))
//           alpha_dot = gdot - d |gdot| alpha
//   twin:   rho = (Kc/sqrt2) <fm - sum f> < (tau - r - eta rho) / Kt >^nt, gdot = rho
//   eps_p_dot = (1 - sum f) sum_s gdot_s m_s + sum_b gdot_b m_b,  v_dot = |gdot|.
// Integration: n_sub classical RK4 steps along the linear strain path of the
// increment (Sec. 3, "explicit ... Runge-Kutta 4th order").
//
// Template parameter NP selects how the regularised rates are solved:
//   NP > 0   eta > 0 and n = nt = NP (compile-time power): table start, branch-free;
//   NP = -1  eta > 0, any real n, nt >= 1 (powers as 2^(p log2 z)): table start, branch-free;
//   NP = 0   anything else (eta = 0 or non-integer exponents): generic per-system solve.
#pragma once

#include <type_traits>

#include "rve_common.cuh"

namespace rve {

// Table 1 (system 9 read as (1 -1 1)[1 1 0]); crystal frame with c/a = 1.
__host__ __device__ __forceinline__ constexpr int sys_n(int s, int c) {
  constexpr int t[16][3] = {{1, 1, -1}, {1, 1, -1}, {1, 1, -1}, {-1, 1, 1}, {-1, 1, 1}, {-1, 1, 1},
                            {1, -1, 1}, {1, -1, 1}, {1, -1, 1}, {1, 1, 1},  {1, 1, 1},  {1, 1, 1},
                            {1, 1, -1}, {-1, 1, 1}, {1, -1, 1}, {1, 1, 1}};
  return t[s][c];
}
__host__ __device__ __forceinline__ constexpr int sys_l(int s, int c) {
  constexpr int t[16][3] = {{0, 1, 1},  {1, 0, 1},  {1, -1, 0},  {0, -1, 1}, {-1, 0, -1}, {-1, -1, 0},
                            {0, 1, 1},  {1, 0, -1}, {1, 1, 0},   {0, 1, -1}, {1, 0, -1},  {1, -1, 0},
                            {1, 1, 2},  {-1, 1, -2}, {1, -1, -2}, {1, 1, -2}};
  return t[s][c];
}

// 1 / (|n| |l|): sqrt(3) sqrt(2) for slip, sqrt(3) sqrt(6) for twins.
template <typename T>
__device__ __forceinline__ T sys_scale(int s) {
  return s < 12 ? T(0.40824829046386301637) : T(0.23570226039551584147);
}

template <typename T>
struct MPState {
  T ep[6];
  T v[16];
  T al[12];
};

template <typename T>
__device__ __forceinline__ void hooke(const MatDev<T>& M, const T* e, T* s) {
  s[0] = M.C11 * e[0] + M.C12 * e[1] + M.C13 * e[2];
  s[1] = M.C12 * e[0] + M.C11 * e[1] + M.C13 * e[2];
  s[2] = M.C13 * (e[0] + e[1]) + M.C33 * e[2];
  s[3] = T(2) * M.C44 * e[3];
  s[4] = T(2) * M.C44 * e[4];
  s[5] = T(2) * M.C66 * e[5];
}

// Integer Schmid coefficients of system s on the six components (11, 22, 33, 23, 13, 12):
// n . x . l = sum_c schmid_k(s, c) x_c for a symmetric x, with schmid_k = n_i l_i on the
// diagonal and n_i l_j + n_j l_i on the shear components.
__host__ __device__ __forceinline__ constexpr int schmid_k(int s, int c) {
  return c == 0   ? sys_n(s, 0) * sys_l(s, 0)
         : c == 1 ? sys_n(s, 1) * sys_l(s, 1)
         : c == 2 ? sys_n(s, 2) * sys_l(s, 2)
         : c == 3 ? sys_n(s, 1) * sys_l(s, 2) + sys_n(s, 2) * sys_l(s, 1)
         : c == 4 ? sys_n(s, 0) * sys_l(s, 2) + sys_n(s, 2) * sys_l(s, 0)
                  : sys_n(s, 0) * sys_l(s, 1) + sys_n(s, 1) * sys_l(s, 0);
}

// sum_c schmid_k(s, c) x_c.  With s a constant (unrolled loops) the zero coefficients
// drop out and unit ones become additions (a product with 0.0 would not fold under IEEE
// rules).
template <typename T>
__device__ __forceinline__ T schmid_sum(int s, const T* x) {
  T r = T(0);
  bool any = false;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const int k = schmid_k(s, c);
    if (k != 0) {
      const T term = k == 1 ? x[c] : (k == -1 ? -x[c] : T(k) * x[c]);
      r = any ? r + term : term;
      any = true;
    }
  }
  return r;
}

// acc_c += schmid_k(s, c) w
template <typename T>
__device__ __forceinline__ void schmid_add(int s, T w, T* acc) {
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const int k = schmid_k(s, c);
    if (k == 1) acc[c] += w;
    else if (k == -1) acc[c] -= w;
    else if (k != 0) acc[c] += T(k) * w;
  }
}

// tau = sigma : m_s = (n . sigma . l) / (|n||l|)
template <typename T>
__device__ __forceinline__ T resolved(int s, const T* g) {
  return sys_scale<T>(s) * schmid_sum<T>(s, g);
}

// Schmid algebra by slip plane.  Every system of Table 1 has a {111} normal n with
// components +-1; systems 3p, 3p+1, 3p+2 and the twin 12+p share plane p.  For such an n and
// any l with n . l = 0 the shear coefficients of schmid_k are the diagonal ones times a sign
// of the plane: n2 l3 + n3 l2 = -n2 n3 (n1 l1), n1 l3 + n3 l1 = -n1 n3 (n2 l2),
// n1 l2 + n2 l1 = -n1 n2 (n3 l3) (from n . l = 0 and n_i^2 = 1).  Hence
//   sum_c schmid_k(s, c) x_c = sum_i (n_i l_i) S_i,  S_i = x_i + sig_i x_(i+3)  (plane sums),
// and sum_s g_s schmid_k(s, c) puts D_i = sum_s (n_i l_i) g_s on component i and sig_i D_i
// on component i + 3.  A slip system has one zero n_i l_i, so its resolved stress is one
// addition of plane sums and a plane's three systems add 3 + 6 terms to a rate sum
// instead of 12; the twins all have n_i l_i = (1, 1, -2).
__host__ __device__ __forceinline__ constexpr int diag_k(int s, int i) { return sys_n(s, i) * sys_l(s, i); }
__host__ __device__ __forceinline__ constexpr int plane_sig(int p, int i) {
  return -sys_n(3 * p, (i + 1) % 3) * sys_n(3 * p, (i + 2) % 3);
}
// s is the first slip system of its plane with a non-zero n_i l_i
__host__ __device__ __forceinline__ constexpr bool first_in_plane(int s, int i) {
  return diag_k(s, i) != 0 && (s % 3 == 0 || (diag_k(s - 1, i) == 0 && (s % 3 == 1 || diag_k(s - 2, i) == 0)));
}
__host__ __device__ constexpr bool schmid_by_plane_holds() {
  for (int s = 0; s < 16; ++s) {
    const int p = s < 12 ? s / 3 : s - 12;
    for (int i = 0; i < 3; ++i)
      if (schmid_k(s, i + 3) != plane_sig(p, i) * diag_k(s, i) || sys_n(s, i) != sys_n(3 * p, i)) return false;
  }
  for (int t = 12; t < 16; ++t)
    if (diag_k(t, 0) != 1 || diag_k(t, 1) != 1 || diag_k(t, 2) != -2) return false;
  return true;
}
static_assert(schmid_by_plane_holds(), "Table 1 systems: plane factorisation of the Schmid sums");

// sum_i diag_k(s, i) S_i (zero coefficients drop out, unit ones are additions)
template <typename T>
__device__ __forceinline__ T plane_sum(int s, const T* S) {
  T r = T(0);
  bool any = false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int k = diag_k(s, i);
    if (k != 0) {
      const T term = k == 1 ? S[i] : (k == -1 ? -S[i] : T(k) * S[i]);
      r = any ? r + term : term;
      any = true;
    }
  }
  return r;
}

// Adds the rate g of slip system s to its plane's sums D; after the plane's last system
// adds D to du (the first plane assigns).
template <typename T>
__device__ __forceinline__ void plane_add(int s, T g, T* D, T* du) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int k = diag_k(s, i);
    if (k != 0) {
      const T term = k == 1 ? g : (k == -1 ? -g : T(k) * g);
      if (first_in_plane(s, i)) D[i] = term;
      else D[i] = D[i] + term;
    }
  }
  if (s % 3 == 2) {
    const int p = s / 3;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T hi = plane_sig(p, i) > 0 ? D[i] : -D[i];
      if (p == 0) {
        du[i] = D[i];
        du[i + 3] = hi;
      } else {
        du[i] = du[i] + D[i];
        du[i + 3] = du[i + 3] + hi;
      }
    }
  }
}

// ---------------------------------------------------------------- powers -------------
// z^n for a small positive integer known at run time (loop).
template <typename T>
__device__ __forceinline__ T ipow(T z, int n) {
  T r = T(1), b = z;
  while (n) {
    if (n & 1) r *= b;
    b *= b;
    n >>= 1;
  }
  return r;
}

// z^n for an integer 1 <= n < 64 without branches (selects over a fixed 6-bit loop).
template <typename T>
__device__ __forceinline__ T ipow_sel(T z, int n) {
  T r = T(1), b = z;
#pragma unroll
  for (int bit = 0; bit < 6; ++bit) {
    const T rb = r * b;
    r = ((n >> bit) & 1) ? rb : r;
    b = b * b;
  }
  return r;
}

// z^N for a compile-time N >= 1 (binary powering unrolled by the compiler).
template <int N, typename T>
__device__ __forceinline__ T cpow(T z) {
  if constexpr (N == 1) {
    return z;
  } else if constexpr (N % 2 == 0) {
    const T h = cpow<N / 2, T>(z);
    return h * h;
  } else {
    return z * cpow<N - 1, T>(z);
  }
}

template <typename T, int NP>
__device__ __forceinline__ T zpow(T z, int n_int) {
  if constexpr (NP > 0) return cpow<NP, T>(z);
  else return ipow_sel<T>(z, n_int);
}

template <typename T>
__device__ __forceinline__ T powT(T z, T n, int n_int) {
  return n_int > 0 ? ipow<T>(z, n_int) : pow(z, n);
}

template <typename T> __device__ __forceinline__ T fast_log2(T x);
template <> __device__ __forceinline__ float fast_log2<float>(float x) { return __log2f(x); }
template <> __device__ __forceinline__ double fast_log2<double>(double x) { return log2(x); }
template <typename T> __device__ __forceinline__ T fast_exp2(T x);
// Float: the hardware approximation (relative error below 2^-22, subnormal results
// flushed to zero), used for Newton starting values and the hardening terms
// exp(-b v) = 2^(-b v log2 e) in (0, 1].
template <> __device__ __forceinline__ float fast_exp2<float>(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
template <> __device__ __forceinline__ double fast_exp2<double>(double x) { return exp2(x); }
// e^x for the hardening terms (x = -b v in [-b v_max, 0]): the float intrinsic is within
// a few ulp there.
template <typename T> __device__ __forceinline__ T fast_exp(T x);
template <> __device__ __forceinline__ float fast_exp<float>(float x) { return __expf(x); }
template <> __device__ __forceinline__ double fast_exp<double>(double x) { return exp(x); }
template <typename T> __device__ __forceinline__ T fast_div(T a, T b);
template <> __device__ __forceinline__ float fast_div<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double fast_div<double>(double a, double b) { return a / b; }
// 1/x for the last Newton correction, which needs only a few correct digits in float
template <typename T> __device__ __forceinline__ T fast_rcp(T x);
template <> __device__ __forceinline__ float fast_rcp<float>(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
template <> __device__ __forceinline__ double fast_rcp<double>(double x) { return 1.0 / x; }

// ---------------------------------------------------------------- rate roots ---------
// The regularised rate rho >= 0 solves rho = P < (a - eta rho) / Kn >^n  (Sec. 4), and
// rho = 0 when a <= 0 or P <= 0.  With z = (a - eta rho)/Kn the root solves
// phi(z) = c z^n + Kn z - a = 0, c = eta P, and rho = P z^n.  Scaling z = zB u with
// zB = (a/c)^(1/n) leaves u^n + beta u - 1 = 0, beta = Kn zB / a, whose root u*(beta)
// depends on x = log2(beta) alone.  log2 u*(x) is tabulated per exponent as kRootIv
// linear pieces over [-kRootSpan, kRootSpan] (the kink of its asymptotes min(0, -x) sits
// on a node); outside that range the end pieces continue along the asymptotes.  The
// interpolated start is within 3e-5 of the root, so a fixed number of Newton steps
// reaches round-off (1 in float, 3 in double) and the solve has no data-dependent
// branch.  Logarithms are base 2.

template <typename T> struct TabNewton;
template <> struct TabNewton<float> { static constexpr int value = 1; };
template <> struct TabNewton<double> { static constexpr int value = 3; };

// Coefficients of the branch-free solve for one class of systems at one RK stage: the
// slip systems (P = 1), or the twins at the stage's prefactor P.  With la = log2 a:
// log2 zB = a1 la + b1, and the table coordinate of x = log2 beta is
// t = (x + kRootSpan) kRootPerUnit - 1/2 = a2 la + b2.  P <= 0 is solved as P = 1 (finite
// dummy arithmetic) and the rate is scaled by Pout = 0.
template <typename T>
struct RootCoef {
  T Pout, c, cn, Kn, Kn_n, a1, b1, a2, b2, nm1;
  T lo;  // argument floor of the packed float solves with a compile-time power (root_floor)
};

template <typename T>
__device__ __forceinline__ RootCoef<T> root_coef(T P, T Kn, T n, T inv_n, T lg_Kn, T eta, T lg_eta, T lg_P) {
  RootCoef<T> q;
  const bool pos = P > T(0);
  q.Pout = pos ? P : T(0);
  q.c = eta * (pos ? P : T(1));
  q.cn = n * q.c;
  q.Kn = Kn;
  q.Kn_n = Kn * inv_n;
  q.a1 = inv_n;
  q.b1 = -(lg_eta + (pos ? lg_P : T(0))) * inv_n;
  q.a2 = (inv_n - T(1)) * T(kRootPerUnit);
  q.b2 = (lg_Kn + q.b1 + T(kRootSpan)) * T(kRootPerUnit) - T(0.5);
  q.nm1 = n - T(1);
  q.lo = T(0);
  return q;
}

// The argument whose table coordinate is kRootIv - 1.25, i.e. 3/4 of an interval inside the
// table's upper end (a2 < 0 for n > 1: larger arguments map to smaller coordinates).  The
// packed solves with a compile-time power floor their arguments here, so that their table
// index needs a lower clamp only.  At this argument the root sits on the Norton asymptote
// 2^16 below the kink, and the rate (a/eta) u*^n is below 2^-160 whenever eta >= K (the
// host selects this variant only then), so it rounds to exactly 0 in float: every argument
// at or below the floor -- inactive systems (a <= 0), NaN, and the positive arguments whose
// exact rate underflows -- returns the masked form's value 0.
__device__ __forceinline__ float root_floor(const RootCoef<float>& q) {
  return fast_exp2<float>(__fdividef(float(kRootIv) - 1.25f - q.b2, q.a2));
}

// z^(n-1) for the table-started Newton steps (z > 0): a compile-time product for NP > 0,
// 2^((n-1) log2 z) for a real exponent (NP = -1; in float the hardware log2 / exp2, whose
// relative error stays far below the 2e-4 the float path is held to).
template <typename T, int NP>
__device__ __forceinline__ T root_zn1(T z, const RootCoef<T>& q, int n_int) {
  if constexpr (NP > 0) return cpow<NP - 1, T>(z);
  else if constexpr (NP < 0) return fast_exp2<T>(q.nm1 * fast_log2<T>(z));
  else return ipow_sel<T>(z, n_int - 1);
}

// Table interval of the coordinate t: floor(t + 1/2) clamped to [0, kRootIv - 1] (any t,
// NaN included, gives an index inside the table).  In float the rounding happens at the
// 1.5 * 2^23 binade, where the spacing is 1, keeping it off the conversion pipe.
template <typename T> __device__ __forceinline__ int root_interval(T t);
template <> __device__ __forceinline__ int root_interval<float>(float t) {
  const float m = t + 12582912.0f;
  const int i = __float_as_int(m) - 0x4B400000;
  return min(max(i, 0), kRootIv - 1);
}
template <> __device__ __forceinline__ int root_interval<double>(double t) {
  double u = t + 0.5;
  u = u > 0.0 ? u : 0.0;
  u = u < double(kRootIv - 1) ? u : double(kRootIv - 1);
  return (int)u;
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Newton steps from z and the rate.  All but the last step are full; the last one is
// folded into the power: with dz = -phi/phi', phi = z (c z^(n-1) + Kn) - a and
// phi' = n (c z^(n-1) + Kn/n), rho = P (z + dz)^n = P z^(n-1) (z + n dz) + O(dz^2);
// |dz/z| < 3e-5 from the table start, so the dropped term n(n-1)/2 (dz/z)^2 < 4e-8 (n = 10)
// is below float round-off (in double two full steps come first).
template <typename T, int NP>
__device__ __forceinline__ T root_newton(T z, T aa, const RootCoef<T>& q, int n_int) {
#pragma unroll
  for (int it = 0; it + 1 < TabNewton<T>::value; ++it) {
    const T zn1 = root_zn1<T, NP>(z, q, n_int);
    const T phi = (q.c * zn1) * z + (q.Kn * z - aa);
    z = z - fast_div<T>(phi, q.cn * zn1 + q.Kn);
  }
  const T zn1 = root_zn1<T, NP>(z, q, n_int);
  const T phi = z * (q.c * zn1 + q.Kn) - aa;
  const T r = fast_rcp<T>(q.c * zn1 + q.Kn_n);  // = n / phi'
  return q.Pout * (zn1 * (z - phi * r));
}

// Branch-free solve (eta > 0, integer exponent): inactive systems run the same arithmetic
// on a dummy positive argument and return 0, so all systems of a stage form one basic
// block the compiler can interleave.  tab: kRootIv (a_i, b_i) pairs, log2 u* = a_i + b_i t.
template <typename T, int NP>
__device__ __forceinline__ T reg_rate_tab(T a, const RootCoef<T>& q, int n_int, const T* tab) {
  const bool on = a > T(0);
  const T aa = on ? a : T(1);
  const T la = fast_log2<T>(aa);
  const T lzB = la * q.a1 + q.b1;
  const T t = la * q.a2 + q.b2;
  const auto ab = reinterpret_cast<const typename Vec2<T>::type*>(tab)[root_interval<T>(t)];
  const T z = fast_exp2<T>(lzB + (ab.x + ab.y * t));
  const T rho = root_newton<T, NP>(z, aa, q, n_int);
  return on ? rho : T(0);
}

// The same for the slip systems, whose coefficients do not depend on the stage (P = 1):
// their table holds log2 z0 = alpha_i + beta_i la directly (alpha_i = b1 + a_i + b_i b2,
// beta_i = a1 + b_i a2, built on the host for the material's K, n and eta).
template <typename T, int NP>
__device__ __forceinline__ T reg_rate_slip(T a, const RootCoef<T>& q, int n_int, const T* tab) {
  const bool on = a > T(0);
  const T aa = on ? a : T(1);
  const T la = fast_log2<T>(aa);
  const T t = la * q.a2 + q.b2;
  const auto ab = reinterpret_cast<const typename Vec2<T>::type*>(tab)[root_interval<T>(t)];
  const T z = fast_exp2<T>(ab.x + ab.y * la);
  const T rho = root_newton<T, NP>(z, aa, q, n_int);
  return on ? rho : T(0);
}

// The float solves of two systems of one class at once, on packed two-lane FP32
// arithmetic (one issue slot per pair of FMAs or products).  Each lane performs the
// operations of reg_rate_slip / reg_rate_tab in the same order and rounding; the
// logarithms, exponentials and reciprocals stay per lane.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

template <int NP>
__device__ __forceinline__ float2 root_zn1_2(float2 z, const RootCoef<float>& q, int n_int) {
  if constexpr (NP > 0) {
    // z^(NP-1) by the binary powering of cpow<NP - 1>, both lanes at once
    float2 r = z;
    constexpr int e = NP - 1;
    if constexpr (e == 9) {
      const float2 h2 = __fmul2_rn(z, z), h4 = __fmul2_rn(h2, h2), h8 = __fmul2_rn(h4, h4);
      r = __fmul2_rn(z, h8);
    } else {
      r = make_float2(cpow<NP - 1, float>(z.x), cpow<NP - 1, float>(z.y));
    }
    return r;
  } else {
    const float2 l = __fmul2_rn(f2(q.nm1), make_float2(fast_log2<float>(z.x), fast_log2<float>(z.y)));
    return make_float2(fast_exp2<float>(l.x), fast_exp2<float>(l.y));
  }
}

// UNIT_P: the slip systems' prefactor P = 1 (no final scaling).
template <int NP, bool UNIT_P = false>
__device__ __forceinline__ float2 root_newton2(float2 z, float2 aa, const RootCoef<float>& q, int n_int) {
  const float2 zn1 = root_zn1_2<NP>(z, q, n_int);
  const float2 phi = __ffma2_rn(z, __ffma2_rn(f2(q.c), zn1, f2(q.Kn)), make_float2(-aa.x, -aa.y));
  const float2 den = __ffma2_rn(f2(q.c), zn1, f2(q.Kn_n));
  const float2 r = make_float2(fast_rcp<float>(den.x), fast_rcp<float>(den.y));
  const float2 w = __ffma2_rn(make_float2(-phi.x, -phi.y), r, z);
  if constexpr (UNIT_P) return __fmul2_rn(zn1, w);
  else return __fmul2_rn(f2(q.Pout), __fmul2_rn(zn1, w));
}

// With a compile-time power (NP = n = nt = 10) an inactive system (a <= 0, or NaN) is solved
// at the floor q.lo (root_floor) instead of being masked: its rate rounds to exactly 0 --
// the masked form's value -- while one min replaces a compare and two selects per system,
// and the floor bounds the table coordinate from above.  A real exponent near 1 would not
// underflow, so NP = -1 keeps the mask.
template <int NP>
__device__ __forceinline__ float2 rate_arg2(float2 a, float lo) {
  if constexpr (NP > 0) return make_float2(fmaxf(a.x, lo), fmaxf(a.y, lo));
  else return make_float2(a.x > 0.f ? a.x : 1.f, a.y > 0.f ? a.y : 1.f);
}

// Table entries at the coordinates t of a pair.  NP > 0: t <= kRootIv - 1.25 (floored
// arguments), so only the lower clamp remains; it is taken in float on t rounded at the
// 1.5 * 2^23 binade (any t, -inf included, gives an index in [0, kRootIv - 1]), and the
// binade's offset folds into the table address.
template <int NP>
__device__ __forceinline__ void tab_pair(float2 t, const float* tab, float2& ab0, float2& ab1) {
  const float2* tb = reinterpret_cast<const float2*>(tab);
  if constexpr (NP > 0) {
    const float2 m = __fadd2_rn(t, f2(12582912.0f));
    ab0 = tb[__float_as_int(fmaxf(m.x, 12582912.0f)) - 0x4B400000];
    ab1 = tb[__float_as_int(fmaxf(m.y, 12582912.0f)) - 0x4B400000];
  } else {
    ab0 = tb[root_interval<float>(t.x)];
    ab1 = tb[root_interval<float>(t.y)];
  }
}
template <int NP>
__device__ __forceinline__ float2 rate_out2(float2 a, float2 rho) {
  if constexpr (NP > 0) return rho;
  else return make_float2(a.x > 0.f ? rho.x : 0.f, a.y > 0.f ? rho.y : 0.f);
}

template <int NP>
__device__ __forceinline__ float2 reg_rate_slip2(float2 a, const RootCoef<float>& q, int n_int, const float* tab) {
  const float2 aa = rate_arg2<NP>(a, q.lo);
  const float2 la = make_float2(fast_log2<float>(aa.x), fast_log2<float>(aa.y));
  const float2 t = __ffma2_rn(la, f2(q.a2), f2(q.b2));
  float2 ab0, ab1;
  tab_pair<NP>(t, tab, ab0, ab1);
  // one FMA per lane: the two systems' table entries are not an operand pair
  const float2 ex = make_float2(fmaf(ab0.y, la.x, ab0.x), fmaf(ab1.y, la.y, ab1.x));
  const float2 z = make_float2(fast_exp2<float>(ex.x), fast_exp2<float>(ex.y));
  const float2 rho = root_newton2<NP, true>(z, aa, q, n_int);
  return rate_out2<NP>(a, rho);
}

template <int NP>
__device__ __forceinline__ float2 reg_rate_tab2(float2 a, const RootCoef<float>& q, int n_int, const float* tab) {
  const float2 aa = rate_arg2<NP>(a, q.lo);
  const float2 la = make_float2(fast_log2<float>(aa.x), fast_log2<float>(aa.y));
  const float2 lzB = __ffma2_rn(la, f2(q.a1), f2(q.b1));
  const float2 t = __ffma2_rn(la, f2(q.a2), f2(q.b2));
  float2 ab0, ab1;
  tab_pair<NP>(t, tab, ab0, ab1);
  const float2 ex = __fadd2_rn(lzB, make_float2(fmaf(ab0.y, t.x, ab0.x), fmaf(ab1.y, t.y, ab1.x)));
  const float2 z = make_float2(fast_exp2<float>(ex.x), fast_exp2<float>(ex.y));
  const float2 rho = root_newton2<NP>(z, aa, q, n_int);
  return rate_out2<NP>(a, rho);
}

// Generic solve (any eta >= 0 and exponent n >= 1): per-system branch, a smooth-minimum
// start u0 = (1 + beta^m)^(-1/m) of the asymptotes (m makes it exact at beta = 1; within
// 5 % for n >= 1.5) and a fixed Newton count (4 in float, 6 in double).
template <typename T> struct NewtonSteps;
template <> struct NewtonSteps<float> { static constexpr int value = 4; };
template <> struct NewtonSteps<double> { static constexpr int value = 6; };

template <typename T>
__device__ __forceinline__ T reg_rate(T a, T P, T Kn, T n, int n_int, T inv_n, T m, T lg_Kn, T eta, T lg_eta,
                                      T lg_P) {
  if (!(a > T(0)) || !(P > T(0))) return T(0);
  if (!(eta > T(0))) return P * powT<T>(a / Kn, n, n_int);
  const T c = eta * P;
  const T la = fast_log2<T>(a);
  const T lzB = (la - lg_eta - lg_P) * inv_n;
  const T lb = lg_Kn + lzB - la;
  const T L = m * lb;
  const T lu = L > T(0) ? -lb - fast_log2<T>(T(1) + fast_exp2<T>(-L)) / m
                        : -fast_log2<T>(T(1) + fast_exp2<T>(L)) / m;
  T z = fast_exp2<T>(lzB + lu);
#pragma unroll
  for (int it = 0; it < NewtonSteps<T>::value; ++it) {
    const T zn1 = n_int > 0 ? ipow<T>(z, n_int - 1) : pow(z, n - T(1));
    const T phi = c * zn1 * z + Kn * z - a;
    z = z - fast_div<T>(phi, n * c * zn1 + Kn);
  }
  z = z > T(0) ? z : T(0);
  return P * powT<T>(z, n, n_int);
}

// ---------------------------------------------------------------- RK4 stage ----------
// One regularised-rate solve: table start for NP != 0, generic otherwise.
template <typename T, int NP>
__device__ __forceinline__ T stage_rate(const MatDev<T>& M, const RootCoef<T>& q, T a, T P, bool twin, T lg_P,
                                        const T* tab) {
  if constexpr (NP != 0) {
    return twin ? reg_rate_tab<T, NP>(a, q, M.nt_int, tab + kRootTabLen) : reg_rate_slip<T, NP>(a, q, M.n_int, tab);
  } else {
    return twin ? reg_rate<T>(a, P, M.Kt, M.nt, M.nt_int, M.inv_nt, M.smt, M.lg_Kt, M.eta, M.lg_eta, lg_P)
                : reg_rate<T>(a, P, M.K, M.n, M.n_int, M.inv_n, M.sm, M.lg_K, M.eta, M.lg_eta, lg_P);
  }
}

// Packed two-lane solves: float with a table-started solve.
template <typename T, int NP>
constexpr bool kPackedSolve = std::is_same<T, float>::value && NP != 0;

// Two values of a pair of systems (or components).  Float: one packed two-lane FP32
// instruction per operation; double: the scalar expressions.
template <typename T> struct PairT;
template <> struct PairT<float> { using type = float2; };
template <> struct PairT<double> { using type = double2; };
template <typename T> using pair_t = typename PairT<T>::type;

template <typename T>
__device__ __forceinline__ pair_t<T> pmk(T a, T b) {
  pair_t<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ pair_t<T> pfma(pair_t<T> a, pair_t<T> b, pair_t<T> c) {  // a b + c
  if constexpr (std::is_same<T, float>::value) return __ffma2_rn(a, b, c);
  else return pmk<T>(a.x * b.x + c.x, a.y * b.y + c.y);
}
template <typename T>
__device__ __forceinline__ pair_t<T> pmul(pair_t<T> a, pair_t<T> b) {
  if constexpr (std::is_same<T, float>::value) return __fmul2_rn(a, b);
  else return pmk<T>(a.x * b.x, a.y * b.y);
}
template <typename T>
__device__ __forceinline__ pair_t<T> padd(pair_t<T> a, pair_t<T> b) {
  if constexpr (std::is_same<T, float>::value) return __fadd2_rn(a, b);
  else return pmk<T>(a.x + b.x, a.y + b.y);
}

// Evaluates the rates at elastic strain e0 + s*de - yt.ep and state yt, adds
// wacc * rates to acc and overwrites yt with y0 + cnext * rates.  FIRST (the first stage of
// a substep, wacc = 1): the input state is y0 and acc is assigned the rates, so neither the
// copy yt = y0 nor the zeroing of acc is needed.
// tab: the rate-root tables (slip systems' at 0, twin exponent's at kRootTabLen), NP != 0 only.
// The systems go in pairs (k, k + 1): both are resolved, solved and folded into acc / yt
// before the next pair (yt.v and yt.al of a pair are read before they are overwritten;
// the hardening terms use the stage's yt.v, computed first).  In float the pair's
// arithmetic runs on packed two-lane instructions.  With NP != 0 the solves are
// branch-free, so the whole stage is one basic block the compiler interleaves; this order
// keeps fewer values live than solving all 16 systems first.
// Rewritten forms (same quantities): with e_k = exp(-b v_k) = 1 - g_k,
//   r_k = r0_k + Q (h_off sum g + (h_diag - h_off) g_k) = (r0_k + Q (h_off (N - sum e) + dq)) - Q dq e_k;
// the slip systems' Schmid scale 1/sqrt6 is folded into the moduli (MatDev C*s, the stress
// itself is not formed), the resolved stresses and the plastic strain rate go through the
// plane sums (plane_sum, plane_add), and the rate sums are scaled once at the end.
template <typename T, int NP, bool FIRST = false>
__device__ __forceinline__ void rk_stage(const MatDev<T>& M, const T* e0, const T* de, T s,
                                         const MPState<T>& y0, MPState<T>& yt, MPState<T>& acc, T wacc,
                                         T cnext, const T* tab) {
  constexpr double kLog2e = 1.44269504088896340736;
  // the stage's input state: y0 in the first stage (so yt needs no copy of it), yt after
  const MPState<T>& yin = FIRST ? y0 : yt;
  // e = e0 + s de - eps_p and the slip-scaled stress ss = C : e / sqrt6 (MatDev's C*s)
  T e[6], ss[6];
  if constexpr (std::is_same<T, float>::value) {
#pragma unroll
    for (int c = 0; c < 6; c += 2) {
      const pair_t<T> ec = pfma<T>(pmk<T>(s, s), pmk<T>(de[c], de[c + 1]), pmk<T>(e0[c], e0[c + 1]));
      e[c] = ec.x - yin.ep[c];
      e[c + 1] = ec.y - yin.ep[c + 1];
    }
    const pair_t<T> s01 = pfma<T>(pmk<T>(M.C13s, M.C13s), pmk<T>(e[2], e[2]),
                                  pfma<T>(pmk<T>(M.C12s, M.C11s), pmk<T>(e[1], e[1]),
                                          pmul<T>(pmk<T>(M.C11s, M.C12s), pmk<T>(e[0], e[0]))));
    const pair_t<T> s45 = pmul<T>(pmk<T>(M.C44s2, M.C66s2), pmk<T>(e[4], e[5]));
    ss[0] = s01.x;
    ss[1] = s01.y;
    ss[2] = M.C13s * (e[0] + e[1]) + M.C33s * e[2];
    ss[3] = M.C44s2 * e[3];
    ss[4] = s45.x;
    ss[5] = s45.y;
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = e0[c] + s * de[c] - yin.ep[c];
    ss[0] = M.C11s * e[0] + M.C12s * e[1] + M.C13s * e[2];
    ss[1] = M.C12s * e[0] + M.C11s * e[1] + M.C13s * e[2];
    ss[2] = M.C13s * (e[0] + e[1]) + M.C33s * e[2];
    ss[3] = M.C44s2 * e[3];
    ss[4] = M.C44s2 * e[4];
    ss[5] = M.C66s2 * e[5];
  }
  T ex[16];
  const T cb_s = -M.b_s * T(kLog2e), cb_t = -M.b_b * T(kLog2e);
  // sums of the hardening terms and twin slips, even and odd systems in the two lanes
  pair_t<T> es2 = pmk<T>(T(0), T(0)), et2 = pmk<T>(T(0), T(0)), vt2 = pmk<T>(T(0), T(0));
#pragma unroll
  for (int k = 0; k < 12; k += 2) {
    const pair_t<T> p = pmul<T>(pmk<T>(cb_s, cb_s), pmk<T>(yin.v[k], yin.v[k + 1]));
    ex[k] = fast_exp2<T>(p.x);
    ex[k + 1] = fast_exp2<T>(p.y);
    es2 = padd<T>(es2, pmk<T>(ex[k], ex[k + 1]));
  }
#pragma unroll
  for (int k = 12; k < 16; k += 2) {
    const pair_t<T> p = pmul<T>(pmk<T>(cb_t, cb_t), pmk<T>(yin.v[k], yin.v[k + 1]));
    ex[k] = fast_exp2<T>(p.x);
    ex[k + 1] = fast_exp2<T>(p.y);
    et2 = padd<T>(et2, pmk<T>(ex[k], ex[k + 1]));
    vt2 = padd<T>(vt2, pmk<T>(yin.v[k], yin.v[k + 1]));
  }
  const T Es = es2.x + es2.y, Et = et2.x + et2.y, vtw = vt2.x + vt2.y;
  const T ftot = T(1.41421356237309504880) * vtw;
  const T wslip = T(1) - ftot;
  T fm_left = M.fm - ftot;
  fm_left = fm_left > T(0) ? fm_left : T(0);
  const T Ptw = (M.Kc * T(0.70710678118654752440)) * fm_left;
  const T lg_Ptw = fast_log2<T>(Ptw > T(0) ? Ptw : T(1));
  const T dq = M.h_diag - M.h_off;
  const T Qdq_s = M.Q_s * dq, Qdq_t = M.Q_b * dq;
  const T Rb_s = M.Q_s * (M.h_off * (T(12) - Es) + dq);
  const T Rb_t = M.Q_b * (M.h_off * (T(4) - Et) + dq);
  // initial resistance plus the stage's common hardening term per kind of system (Table 1:
  // systems 3, 6, 9 and 12 ordinary, the other slip systems superdislocations; one value for
  // the twins), as the host fills M.r0
  const T rb_sup = M.r0[0] + Rb_s, rb_ord = M.r0[2] + Rb_s, rb_tw = M.r0[12] + Rb_t;
  RootCoef<T> qs, qt;
  if constexpr (NP != 0) {
    qs = root_coef<T>(T(1), M.K, M.n, M.inv_n, M.lg_K, M.eta, M.lg_eta, T(0));
    qt = root_coef<T>(Ptw, M.Kt, M.nt, M.inv_nt, M.lg_Kt, M.eta, M.lg_eta, lg_Ptw);
    if constexpr (kPackedSolve<T, NP> && NP > 0) {
      qs.lo = root_floor(qs);
      qt.lo = root_floor(qt);
    }
  }
  // plane sums of the slip-scaled stress (plane_sum)
  T S[4][3];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int i = 0; i < 3; ++i) S[p][i] = plane_sig(p, i) > 0 ? ss[i] + ss[i + 3] : ss[i] - ss[i + 3];
  T du_s[6], D[3];
  // the systems in pairs: both driving forces, both rates (packed solve in float), then
  // each system folded into acc / yt
#pragma unroll
  for (int k = 0; k < 12; k += 2) {
    const pair_t<T> alk = pmk<T>(yin.al[k], yin.al[k + 1]);
    const pair_t<T> tk = pfma<T>(pmk<T>(-M.c, -M.c), alk,
                                 pmk<T>(plane_sum<T>(k, S[k / 3]), plane_sum<T>(k + 1, S[(k + 1) / 3])));
    const pair_t<T> rr = pfma<T>(pmk<T>(-Qdq_s, -Qdq_s), pmk<T>(ex[k], ex[k + 1]),
                                 pmk<T>(k % 3 == 2 ? rb_ord : rb_sup, (k + 1) % 3 == 2 ? rb_ord : rb_sup));
    const T tek0 = tk.x, tek1 = tk.y;
    const T ak0 = fabs(tek0) - rr.x;
    const T ak1 = fabs(tek1) - rr.y;
    T rk2[2];
    if constexpr (kPackedSolve<T, NP>) {
      const float2 r = reg_rate_slip2<NP>(make_float2(ak0, ak1), qs, M.n_int, tab);
      rk2[0] = r.x;
      rk2[1] = r.y;
    } else {
      rk2[0] = stage_rate<T, NP>(M, qs, ak0, T(1), false, T(0), tab);
      rk2[1] = stage_rate<T, NP>(M, qs, ak1, T(1), false, T(0), tab);
    }
    const T gd0 = copysign(rk2[0], tek0);  // rk = 0 unless |tek| > r > 0
    const T gd1 = copysign(rk2[1], tek1);
    plane_add<T>(k, gd0, D, du_s);
    plane_add<T>(k + 1, gd1, D, du_s);
    const pair_t<T> rk = pmk<T>(rk2[0], rk2[1]);
    const pair_t<T> drk = pmul<T>(pmk<T>(-M.d, -M.d), rk);
    const pair_t<T> ald = pfma<T>(drk, alk, pmk<T>(gd0, gd1));  // gd - d rk alpha
    const pair_t<T> wa = pmk<T>(wacc, wacc), cn = pmk<T>(cnext, cnext);
    const pair_t<T> av = FIRST ? rk : pfma<T>(wa, rk, pmk<T>(acc.v[k], acc.v[k + 1]));
    const pair_t<T> yv = pfma<T>(cn, rk, pmk<T>(y0.v[k], y0.v[k + 1]));
    const pair_t<T> aa = FIRST ? ald : pfma<T>(wa, ald, pmk<T>(acc.al[k], acc.al[k + 1]));
    const pair_t<T> ya = pfma<T>(cn, ald, pmk<T>(y0.al[k], y0.al[k + 1]));
    acc.v[k] = av.x;
    acc.v[k + 1] = av.y;
    yt.v[k] = yv.x;
    yt.v[k + 1] = yv.y;
    acc.al[k] = aa.x;
    acc.al[k + 1] = aa.y;
    yt.al[k] = ya.x;
    yt.al[k + 1] = ya.y;
  }
  // twins: the twin rates g_t enter the diagonal components as (G, G, -2 G), G = sum g_t,
  // and component i + 3 as H_i = sum_t sig_i(plane of t) g_t (times -2 for i = 2)
  T G = T(0), H[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int k = 12; k < 16; k += 2) {
    const pair_t<T> rr = pfma<T>(pmk<T>(-Qdq_t, -Qdq_t), pmk<T>(ex[k], ex[k + 1]),
                                 pmk<T>(rb_tw, rb_tw));
    // 1/(|n||l|) of a twin is (1/sqrt3) times the slip systems' scale in ss
    constexpr T kTw = T(0.57735026918962576451);
    const T ak0 = kTw * plane_sum<T>(k, S[k - 12]) - rr.x;
    const T ak1 = kTw * plane_sum<T>(k + 1, S[k - 11]) - rr.y;
    T rk2[2];
    if constexpr (kPackedSolve<T, NP>) {
      const float2 r = reg_rate_tab2<NP>(make_float2(ak0, ak1), qt, M.nt_int, tab + kRootTabLen);
      rk2[0] = r.x;
      rk2[1] = r.y;
    } else {
      rk2[0] = stage_rate<T, NP>(M, qt, ak0, Ptw, true, lg_Ptw, tab);
      rk2[1] = stage_rate<T, NP>(M, qt, ak1, Ptw, true, lg_Ptw, tab);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int p = k - 12 + j;
      const T g = rk2[j];
      G = p == 0 ? g : G + g;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const T hg = plane_sig(p, i) > 0 ? g : -g;
        H[i] = p == 0 ? hg : H[i] + hg;
      }
    }
    const pair_t<T> rk = pmk<T>(rk2[0], rk2[1]);
    const pair_t<T> av = FIRST ? rk : pfma<T>(pmk<T>(wacc, wacc), rk, pmk<T>(acc.v[k], acc.v[k + 1]));
    const pair_t<T> yv = pfma<T>(pmk<T>(cnext, cnext), rk, pmk<T>(y0.v[k], y0.v[k + 1]));
    acc.v[k] = av.x;
    acc.v[k + 1] = av.y;
    yt.v[k] = yv.x;
    yt.v[k + 1] = yv.y;
  }
  // eps_p rate = (1 - sum f) sum_s gdot_s m_s + sum_b gdot_b m_b, m = scale sym(n x l)
  const T fs = wslip * sys_scale<T>(0);
  const T fsh = T(0.5) * fs;
  const T tsc = sys_scale<T>(12), tsh = T(0.5) * sys_scale<T>(12);
  const T du_t[6] = {G, G, T(-2) * G, H[0], H[1], T(-2) * H[2]};
#pragma unroll
  for (int c = 0; c < 6; c += 2) {
    const pair_t<T> dep = pfma<T>(pmk<T>(c < 3 ? fs : fsh, c + 1 < 3 ? fs : fsh), pmk<T>(du_s[c], du_s[c + 1]),
                                  pmul<T>(pmk<T>(c < 3 ? tsc : tsh, c + 1 < 3 ? tsc : tsh),
                                          pmk<T>(du_t[c], du_t[c + 1])));
    const pair_t<T> ae = FIRST ? dep : pfma<T>(pmk<T>(wacc, wacc), dep, pmk<T>(acc.ep[c], acc.ep[c + 1]));
    const pair_t<T> ye = pfma<T>(pmk<T>(cnext, cnext), dep, pmk<T>(y0.ep[c], y0.ep[c + 1]));
    acc.ep[c] = ae.x;
    acc.ep[c + 1] = ae.y;
    yt.ep[c] = ye.x;
    yt.ep[c + 1] = ye.y;
  }
}

// True when no system can be active anywhere on the increment's strain path with the
// state frozen at t_n: |tau - x| - r (slip) and tau - r (twin) are convex in the path
// parameter, so checking both ends suffices; the exact solution is then "no flow".
template <typename T>
__device__ __forceinline__ bool elastic_increment(const MatDev<T>& M, const T* e0, const T* de,
                                                  const MPState<T>& y) {
  T ea[6], eb[6], sa[6], sb[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    ea[c] = e0[c] - y.ep[c];
    eb[c] = e0[c] + de[c] - y.ep[c];
  }
  hooke<T>(M, ea, sa);
  hooke<T>(M, eb, sb);
  T g[16];
  T Sslip = T(0), Stw = T(0), vtw = T(0);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    g[k] = T(1) - fast_exp<T>(-M.b_s * y.v[k]);
    Sslip += g[k];
  }
#pragma unroll
  for (int k = 12; k < 16; ++k) {
    g[k] = T(1) - fast_exp<T>(-M.b_b * y.v[k]);
    Stw += g[k];
    vtw += y.v[k];
  }
  const T dq = M.h_diag - M.h_off;
  bool quiet = true;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const T x = M.c * y.al[k];
    const T r = M.r0[k] + M.Q_s * (M.h_off * Sslip + dq * g[k]);
    const T a0 = fabs(resolved<T>(k, sa) - x) - r;
    const T a1 = fabs(resolved<T>(k, sb) - x) - r;
    quiet = quiet && !(a0 > T(0)) && !(a1 > T(0));
  }
  const T ftot = T(1.41421356237309504880) * vtw;
  if (M.fm - ftot > T(0)) {
#pragma unroll
    for (int k = 12; k < 16; ++k) {
      const T r = M.r0[k] + M.Q_b * (M.h_off * Stw + dq * g[k]);
      const T a0 = resolved<T>(k, sa) - r;
      const T a1 = resolved<T>(k, sb) - r;
      quiet = quiet && !(a0 > T(0)) && !(a1 > T(0));
    }
  }
  return quiet;
}

// eps_c = R^T eps R for a symmetric tensor in 6-component storage; R row-major.
template <typename T>
__device__ __forceinline__ void to_crystal(const T* R, const T* e, T* out) {
  const T E[3][3] = {{e[0], e[5], e[4]}, {e[5], e[1], e[3]}, {e[4], e[3], e[2]}};
  T A[3][3];  // E R
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) A[i][j] = E[i][0] * R[0 * 3 + j] + E[i][1] * R[1 * 3 + j] + E[i][2] * R[2 * 3 + j];
  // out_ij = sum_k R_ki A_kj
  out[0] = R[0] * A[0][0] + R[3] * A[1][0] + R[6] * A[2][0];
  out[1] = R[1] * A[0][1] + R[4] * A[1][1] + R[7] * A[2][1];
  out[2] = R[2] * A[0][2] + R[5] * A[1][2] + R[8] * A[2][2];
  out[3] = R[1] * A[0][2] + R[4] * A[1][2] + R[7] * A[2][2];
  out[4] = R[0] * A[0][2] + R[3] * A[1][2] + R[6] * A[2][2];
  out[5] = R[0] * A[0][1] + R[3] * A[1][1] + R[6] * A[2][1];
}

// sigma = R sigma_c R^T
template <typename T>
__device__ __forceinline__ void to_sample(const T* R, const T* s, T* out) {
  const T S[3][3] = {{s[0], s[5], s[4]}, {s[5], s[1], s[3]}, {s[4], s[3], s[2]}};
  T B[3][3];  // S R^T : B_ij = sum_k S_ik R_jk
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) B[i][j] = S[i][0] * R[j * 3 + 0] + S[i][1] * R[j * 3 + 1] + S[i][2] * R[j * 3 + 2];
  // out_ij = sum_k R_ik B_kj
  out[0] = R[0] * B[0][0] + R[1] * B[1][0] + R[2] * B[2][0];
  out[1] = R[3] * B[0][1] + R[4] * B[1][1] + R[5] * B[2][1];
  out[2] = R[6] * B[0][2] + R[7] * B[1][2] + R[8] * B[2][2];
  out[3] = R[3] * B[0][2] + R[4] * B[1][2] + R[5] * B[2][2];
  out[4] = R[0] * B[0][2] + R[1] * B[1][2] + R[2] * B[2][2];
  out[5] = R[0] * B[0][1] + R[1] * B[1][1] + R[2] * B[2][1];
}

// Integrates one voxel over the increment [t_n, t_n + dt] (strain eps_n -> eps, sample
// frame) and returns the sample-frame stress at t_n + dt; y is updated in place.
// check: test first whether the increment is elastic and skip the integration if so.  The
// test is a shortcut only: with every rate exactly 0 (inactive systems return 0 in every
// rate-solve variant) the RK4 substeps leave the state bit for bit unchanged, so results do
// not depend on it.  Returns false when the test ran and found the increment elastic.
template <typename T, int NP>
__device__ __forceinline__ bool mc_voxel(const MatDev<T>& M, const T* R, const T* eps_n, const T* eps,
                                         MPState<T>& y, T dt, int nsub, T* sig, const T* tab, bool check = true) {
  T e0[6], e1[6], de[6];
  to_crystal<T>(R, eps_n, e0);
  to_crystal<T>(R, eps, e1);
#pragma unroll
  for (int c = 0; c < 6; ++c) de[c] = e1[c] - e0[c];
  const bool flows = !(check && elastic_increment<T>(M, e0, de, y));
  if (flows) {
    const T h = dt / T(nsub);
    const T inv = T(1) / T(nsub);
    for (int m = 0; m < nsub; ++m) {
      const T s0 = T(m) * inv, sh = (T(m) + T(0.5)) * inv, s1 = (T(m) + T(1)) * inv;
      MPState<T> yt, acc;
      // classical RK4: stages at s0, sh, sh, s1 with weights 1, 2, 2, 1.  The first stage
      // reads y and assigns acc and yt; the other three share one copy of the stage body
      // (not unrolled, which keeps the code compact)
      rk_stage<T, NP, true>(M, e0, de, s0, y, yt, acc, T(1), T(0.5) * h, tab);
#pragma unroll 1
      for (int stg = 1; stg < 4; ++stg) {
        const T s = stg == 3 ? s1 : sh;
        const T wacc = stg == 3 ? T(1) : T(2);
        const T cnext = stg == 1 ? T(0.5) * h : (stg == 2 ? h : T(0));
        rk_stage<T, NP>(M, e0, de, s, y, yt, acc, wacc, cnext, tab);
      }
      const T w = h / T(6);
#pragma unroll
      for (int c = 0; c < 6; ++c) y.ep[c] += w * acc.ep[c];
#pragma unroll
      for (int c = 0; c < 16; ++c) y.v[c] += w * acc.v[c];
#pragma unroll
      for (int c = 0; c < 12; ++c) y.al[c] += w * acc.al[c];
    }
  }
  T ee[6], sc[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) ee[c] = e1[c] - y.ep[c];
  hooke<T>(M, ee, sc);
  to_sample<T>(R, sc, sig);
  return flows;
}

template <typename T>
__device__ __forceinline__ T von_mises6(const T* s) {
  const T p = (s[0] + s[1] + s[2]) / T(3);
  const T a = s[0] - p, b = s[1] - p, c = s[2] - p;
  return sqrt(T(1.5) * (a * a + b * b + c * c + T(2) * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5])));
}

}  // namespace rve
