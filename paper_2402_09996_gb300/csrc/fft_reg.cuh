// Register-resident DFTs and the two-step ("four-step" without the transposes in
// memory) decomposition used by the pencil passes for power-of-two line lengths.
//
// A length N = N1 * N2 transform splits, with n = n1 + N1 n2 and k = k2 + N2 k1, into
//   Y[n1][k2] = sum_{n2} x[n1 + N1 n2] W_N2^(n2 k2)      (N1 DFTs of length N2)
//   Y[n1][k2] *= W_N^(n1 k2)                             (twiddles)
//   X[k2 + N2 k1] = sum_{n1} Y[n1][k2] W_N1^(n1 k1)      (N2 DFTs of length N1),
// W_M = e^(SIGN 2 pi i / M) (SIGN = -1 forward, +1 unnormalised inverse).  A thread holds
// one column of either step in registers, so a line moves through shared memory once.
// The short DFTs (2, 4, 8, 16) use the same split recursively with radix-4 butterflies
// and constant twiddles.
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

// In-place DFT of R values in natural order (R = 1, 2, 4, 8, 16).
template <typename T, int SIGN, int R>
__device__ __forceinline__ void dft_reg(C2<T>* v) {
  if constexpr (R == 2) {
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

// The split used for each power-of-two line length: N1 threads per line in the first step
// (N2 values each), N2 columns per line in the second (N1 values each).
template <int N> struct PencilSplit { static constexpr int N1 = 0, N2 = 0; };
template <> struct PencilSplit<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct PencilSplit<128> { static constexpr int N1 = 8, N2 = 16; };
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
