// Batched complex FFTs held in shared memory: self-sorting Stockham passes of
// radix 4, 2, 3 and 5 (Stockham autosort formulation as in Govindaraju et al.,
// "High performance discrete Fourier transforms on graphics processors", SC 2008).
//
// A CTA transforms `nseq` sequences of length n, sequence q starting at q*stride
// (stride >= n; n + 1 avoids shared-memory bank conflicts in transposed loads) in
// buffer `a`; `b` is scratch of the same size.  Every stage reads one
// buffer and writes the other; the function returns the buffer that holds the
// result.  SIGN = -1 is the forward transform (kernel e^{-2 pi i k m / n}),
// SIGN = +1 the unnormalised inverse.  `tw` holds e^{-2 pi i m / n}, m < n.
#pragma once

#include "rve_common.cuh"

namespace rve {

template <typename T, int SIGN>
__device__ __forceinline__ C2<T> mul_i(C2<T> a) {
  // SIGN * i * a
  return (SIGN > 0) ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

template <typename T, int SIGN, int R>
__device__ __forceinline__ void small_dft(C2<T>* v) {
  if (R == 2) {
    C2<T> a = v[0], b = v[1];
    v[0] = cadd<T>(a, b);
    v[1] = csub<T>(a, b);
  } else if (R == 4) {
    C2<T> t0 = cadd<T>(v[0], v[2]);
    C2<T> t1 = csub<T>(v[0], v[2]);
    C2<T> t2 = cadd<T>(v[1], v[3]);
    C2<T> t3 = mul_i<T, SIGN>(csub<T>(v[1], v[3]));
    v[0] = cadd<T>(t0, t2);
    v[2] = csub<T>(t0, t2);
    v[1] = cadd<T>(t1, t3);
    v[3] = csub<T>(t1, t3);
  } else if (R == 3) {
    const T h = T(0.86602540378443864676);  // sin(2 pi / 3)
    C2<T> s = cadd<T>(v[1], v[2]);
    C2<T> d = mul_i<T, SIGN>(cscale<T>(csub<T>(v[1], v[2]), h));
    C2<T> m = csub<T>(v[0], cscale<T>(s, T(0.5)));
    v[0] = cadd<T>(v[0], s);
    v[1] = cadd<T>(m, d);
    v[2] = csub<T>(m, d);
  } else if (R == 5) {
    const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);
    const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);
    C2<T> s14 = cadd<T>(v[1], v[4]), d14 = csub<T>(v[1], v[4]);
    C2<T> s23 = cadd<T>(v[2], v[3]), d23 = csub<T>(v[2], v[3]);
    C2<T> a0 = v[0];
    C2<T> p1 = mk<T>(a0.x + c1 * s14.x + c2 * s23.x, a0.y + c1 * s14.y + c2 * s23.y);
    C2<T> p2 = mk<T>(a0.x + c2 * s14.x + c1 * s23.x, a0.y + c2 * s14.y + c1 * s23.y);
    C2<T> q1 = mul_i<T, SIGN>(mk<T>(s1 * d14.x + s2 * d23.x, s1 * d14.y + s2 * d23.y));
    C2<T> q2 = mul_i<T, SIGN>(mk<T>(s2 * d14.x - s1 * d23.x, s2 * d14.y - s1 * d23.y));
    v[0] = mk<T>(a0.x + s14.x + s23.x, a0.y + s14.y + s23.y);
    v[1] = cadd<T>(p1, q1);
    v[4] = csub<T>(p1, q1);
    v[2] = cadd<T>(p2, q2);
    v[3] = csub<T>(p2, q2);
  }
}

// floor(x / d) for x, d < 2^16 with m = ceil(2^32 / d) (d >= 2): x m / 2^32 exceeds x / d
// by less than x / 2^32 < 1/d, which cannot carry past the next integer.
__device__ __forceinline__ unsigned div_small(unsigned x, unsigned d, unsigned m) {
  return d == 1u ? x : __umulhi(x, m);
}
__device__ __forceinline__ unsigned recip_small(unsigned d) { return d > 1u ? 0xFFFFFFFFu / d + 1u : 0u; }

template <typename T, int SIGN, int R>
__device__ __forceinline__ void stockham_stage(const C2<T>* __restrict__ x, C2<T>* __restrict__ y,
                                               int n, int nseq, int stride, int Ns,
                                               const C2<T>* __restrict__ tw, int tid, int nthr) {
  const int nb = n / R;        // butterflies per sequence
  const int tstride = n / (Ns * R);
  const int total = nseq * nb;
  // the butterfly index splits by multiply-high reciprocals (exact below 2^16), else by division
  const bool small = total < 65536;
  const unsigned m_nb = recip_small((unsigned)nb), m_ns = recip_small((unsigned)Ns);
  for (int w = tid; w < total; w += nthr) {
    const int q = small ? (int)div_small((unsigned)w, (unsigned)nb, m_nb) : w / nb;
    const int j = w - q * nb;
    const int jd = small ? (int)div_small((unsigned)j, (unsigned)Ns, m_ns) : j / Ns;
    const int k = j - jd * Ns;
    const C2<T>* xs = x + q * stride;
    C2<T>* ys = y + q * stride;
    C2<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      C2<T> a = xs[j + r * nb];
      if (r > 0 && k > 0) {
        C2<T> t = tw[r * k * tstride];
        a = (SIGN < 0) ? cmul<T>(a, t) : cmulc<T>(a, t);
      }
      v[r] = a;
    }
    small_dft<T, SIGN, R>(v);
    const int base = jd * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) ys[base + r * Ns] = v[r];
  }
}

// Runs all stages; must be called by every thread of the CTA (contains barriers).
template <typename T, int SIGN>
__device__ C2<T>* smem_fft(C2<T>* a, C2<T>* b, const FftDim& d, int nseq, int stride, const C2<T>* tw,
                           int tid, int nthr) {
  int Ns = 1;
  for (int s = 0; s < d.nst; ++s) {
    const int R = d.radix[s];
    if (R == 4) stockham_stage<T, SIGN, 4>(a, b, d.n, nseq, stride, Ns, tw, tid, nthr);
    else if (R == 2) stockham_stage<T, SIGN, 2>(a, b, d.n, nseq, stride, Ns, tw, tid, nthr);
    else if (R == 3) stockham_stage<T, SIGN, 3>(a, b, d.n, nseq, stride, Ns, tw, tid, nthr);
    else stockham_stage<T, SIGN, 5>(a, b, d.n, nseq, stride, Ns, tw, tid, nthr);
    Ns *= R;
    __syncthreads();
    C2<T>* t = a;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace rve
