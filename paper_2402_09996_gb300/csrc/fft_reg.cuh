// Register-resident DFTs and the two-step ("four-step" without the transposes in
// memory) decomposition used by the pencil passes for the line lengths 64, 96, 128, 160
// and 256.
//
// A length N = N1 * N2 transform splits, with n = n1 + N1 n2 and k = k2 + N2 k1, into
//   Y[n1][k2] = sum_{n2} x[n1 + N1 n2] W_N2^(n2 k2)      (N1 DFTs of length N2)
//   Y[n1][k2] *= W_N^(n1 k2)                             (twiddles)
//   X[k2 + N2 k1] = sum_{n1} Y[n1][k2] W_N1^(n1 k1)      (N2 DFTs of length N1),
// W_M = e^(SIGN 2 pi i / M) (SIGN = -1 forward, +1 unnormalised inverse).  A thread holds
// one column of either step in registers, so a line moves through shared memory once.
// The short DFTs use the same split recursively: 8 and 16 with radix-4 butterflies, 10 =
// 2 * 5 and 12 = 4 * 3 with the radix-2/3/4/5 butterflies of fft_smem.cuh; all their
// twiddles are compile-time constants.
#pragma once

#include "fft_smem.cuh"

namespace rve {

// cos and sin of 2 pi e / 16, e = 0 .. 15
__device__ __forceinline__ constexpr double cos16(int e) {
  constexpr double c[16] = {1.0,
                            0.92387953251128675613,
                            0.70710678118654752440,
                            0.38268343236508977173,
                            0.0,
                            -0.38268343236508977173,
                            -0.70710678118654752440,
                            -0.92387953251128675613,
                            -1.0,
                            -0.92387953251128675613,
                            -0.70710678118654752440,
                            -0.38268343236508977173,
                            0.0,
                            0.38268343236508977173,
                            0.70710678118654752440,
                            0.92387953251128675613};
  return c[e & 15];
}
__device__ __forceinline__ constexpr double sin16(int e) { return cos16(e - 4); }

// cos and sin of 2 pi e / R for integers e, R (R > 0), evaluated at compile time: the
// rational angle is reduced exactly to a quarter turn q and a remainder in [0, pi/4] (by
// the complement when above pi/4), where the Taylor series of sin and cos converge to
// double precision in a dozen terms.
constexpr double kPi = 3.14159265358979323846;
__host__ __device__ constexpr double series_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 12; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double series_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 12; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
struct CosSin {
  double c, s;
};
__host__ __device__ constexpr CosSin unit_root(int e, int R) {
  e %= R;
  if (e < 0) e += R;
  const int q = 4 * e / R, r = 4 * e - q * R;  // angle = (pi/2) (q + r / R), 0 <= r < R
  double c = 0.0, s = 0.0;
  if (2 * r <= R) {
    const double t = 0.5 * kPi * r / R;
    c = series_cos(t);
    s = series_sin(t);
  } else {
    const double t = 0.5 * kPi * (R - r) / R;
    c = series_sin(t);
    s = series_cos(t);
  }
  if (q == 0) return CosSin{c, s};
  if (q == 1) return CosSin{-s, c};
  if (q == 2) return CosSin{-c, -s};
  return CosSin{s, -c};
}

// a * W_R^E, W_R = e^(SIGN 2 pi i / R), E a compile-time constant: factors 1, -1 and +-i
// take no multiplication.
template <typename T, int SIGN, int R, int E>
__device__ __forceinline__ C2<T> rot_root(C2<T> a) {
  constexpr int e = ((E % R) + R) % R;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (2 * e == R) {
    return mk<T>(-a.x, -a.y);
  } else if constexpr (4 * e == R) {
    return mul_i<T, SIGN>(a);
  } else if constexpr (4 * e == 3 * R) {
    return mul_i<T, -SIGN>(a);
  } else {
    constexpr CosSin w = unit_root(e, R);
    const T c = T(w.c), s = T(SIGN * w.s);
    return mk<T>(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

// a * W_R^e, W_R = e^(SIGN 2 pi i / R), R | 16, e a compile-time constant: the eighth
// roots of unity take additions only where the factor is 1, -1 or +-i.
template <typename T, int SIGN, int R, int E>
__device__ __forceinline__ C2<T> rot_const(C2<T> a) {
  constexpr int e = ((E % R) * (16 / R)) & 15;  // exponent in units of 2 pi / 16
  if constexpr (e == 0) {
    return a;
  } else if constexpr (e == 8) {
    return mk<T>(-a.x, -a.y);
  } else if constexpr (e == 4) {
    return mul_i<T, SIGN>(a);
  } else if constexpr (e == 12) {
    return mul_i<T, -SIGN>(a);
  } else {
    constexpr double cd = cos16(e), sd = SIGN * sin16(e);
    const T c = T(cd), s = T(sd);
    return mk<T>(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

template <typename T, int SIGN, int R, int M, int K>
__device__ __forceinline__ void dft_twiddle_row(C2<T>* b) {
  if constexpr (K < 4) {
    b[K] = rot_const<T, SIGN, R, M * K>(b[K]);
    dft_twiddle_row<T, SIGN, R, M, K + 1>(b);
  }
}

template <typename T, int SIGN, int R>
__device__ __forceinline__ void dft_reg(C2<T>* v);

// w[K] *= W_R^(M K) for K = K0 .. KEND - 1 (compile-time exponents).
template <typename T, int SIGN, int R, int M, int K, int KEND>
__device__ __forceinline__ void twiddle_seq(C2<T>* w) {
  if constexpr (K < KEND) {
    w[K] = rot_root<T, SIGN, R, M * K>(w[K]);
    twiddle_seq<T, SIGN, R, M, K + 1, KEND>(w);
  }
}

// First step of the A * B split for every a (compile-time): the B-point DFT of
// v[a + A b] over b, times W_(AB)^(a kb), into y[a * B + kb].
template <typename T, int SIGN, int A, int B, int a>
__device__ __forceinline__ void mixed_step1(const C2<T>* v, C2<T>* y) {
  if constexpr (a < A) {
    C2<T> w[B];
#pragma unroll
    for (int b = 0; b < B; ++b) w[b] = v[a + A * b];
    dft_reg<T, SIGN, B>(w);
    twiddle_seq<T, SIGN, A * B, a, 0, B>(w);
#pragma unroll
    for (int kb = 0; kb < B; ++kb) y[a * B + kb] = w[kb];
    mixed_step1<T, SIGN, A, B, a + 1>(v, y);
  }
}

// In-place DFT of R = A * B values in natural order: with n = a + A b and k = kb + B ka,
// X[kb + B ka] = sum_a W_A^(a ka) W_R^(a kb) sum_b v[a + A b] W_B^(b kb).
template <typename T, int SIGN, int A, int B>
__device__ __forceinline__ void dft_mixed(C2<T>* v) {
  C2<T> y[A * B];
  mixed_step1<T, SIGN, A, B, 0>(v, y);
#pragma unroll
  for (int kb = 0; kb < B; ++kb) {
    C2<T> u[A];
#pragma unroll
    for (int a = 0; a < A; ++a) u[a] = y[a * B + kb];
    dft_reg<T, SIGN, A>(u);
#pragma unroll
    for (int ka = 0; ka < A; ++ka) v[kb + B * ka] = u[ka];
  }
}

// In-place DFT of R values in natural order (R = 1, 2, 3, 4, 5, 8, 10, 12, 16).
template <typename T, int SIGN, int R>
__device__ __forceinline__ void dft_reg(C2<T>* v) {
  if constexpr (R == 3 || R == 5) {
    small_dft<T, SIGN, R>(v);
  } else if constexpr (R == 10) {
    dft_mixed<T, SIGN, 2, 5>(v);
  } else if constexpr (R == 12) {
    dft_mixed<T, SIGN, 4, 3>(v);
  } else if constexpr (R == 2) {
    const C2<T> a = v[0], b = v[1];
    v[0] = cadd<T>(a, b);
    v[1] = csub<T>(a, b);
  } else if constexpr (R == 4) {
    small_dft<T, SIGN, 4>(v);
  } else if constexpr (R > 4) {
    constexpr int M = R / 4;
    C2<T> b[R];  // b[m * 4 + k2]
#pragma unroll
    for (int m = 0; m < M; ++m) {
      C2<T> a[4] = {v[m], v[m + M], v[m + 2 * M], v[m + 3 * M]};
      small_dft<T, SIGN, 4>(a);
#pragma unroll
      for (int k = 0; k < 4; ++k) b[m * 4 + k] = a[k];
    }
    if constexpr (M == 2) {
      dft_twiddle_row<T, SIGN, R, 1, 0>(b + 4);
    } else if constexpr (M == 4) {
      dft_twiddle_row<T, SIGN, R, 1, 0>(b + 4);
      dft_twiddle_row<T, SIGN, R, 2, 0>(b + 8);
      dft_twiddle_row<T, SIGN, R, 3, 0>(b + 12);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      C2<T> c[M];
#pragma unroll
      for (int m = 0; m < M; ++m) c[m] = b[m * 4 + k];
      dft_reg<T, SIGN, M>(c);
#pragma unroll
      for (int q = 0; q < M; ++q) v[k + 4 * q] = c[q];
    }
  }
}

// The split used for each line length: N1 threads per line in the first step
// (N2 values each), N2 columns per line in the second (N1 values each).
template <int N> struct PencilSplit { static constexpr int N1 = 0, N2 = 0; };
template <> struct PencilSplit<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct PencilSplit<96> { static constexpr int N1 = 8, N2 = 12; };
template <> struct PencilSplit<128> { static constexpr int N1 = 8, N2 = 16; };
template <> struct PencilSplit<160> { static constexpr int N1 = 10, N2 = 16; };
template <> struct PencilSplit<256> { static constexpr int N1 = 16, N2 = 16; };

// First step for the column n1 of one line: v[n2] = x[n1 + N1 n2] in, the twiddled
// Y[n1][k2] out to shared memory at line[k2 * N1 + n1].  tw[e] = e^(-2 pi i e / N).
template <typename T, int SIGN, int N1, int N2>
__device__ __forceinline__ void pencil_step1(C2<T>* v, int n1, C2<T>* line, const C2<T>* tw) {
  dft_reg<T, SIGN, N2>(v);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    C2<T> a = v[k2];
    if (k2 > 0 && n1 > 0) {
      const C2<T> t = tw[n1 * k2];
      a = (SIGN < 0) ? cmul<T>(a, t) : cmulc<T>(a, t);
    }
    line[k2 * N1 + n1] = a;
  }
}

// Second step for the column k2: v[n1] = Y[n1][k2] read from shared memory, and out
// v[k1] = X[k2 + N2 k1].
template <typename T, int SIGN, int N1, int N2>
__device__ __forceinline__ void pencil_step2(C2<T>* v, int k2, const C2<T>* line) {
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) v[n1] = line[k2 * N1 + n1];
  dft_reg<T, SIGN, N1>(v);
}

}  // namespace rve
