// Kernels of one fixed-point iteration of the Green-operator solver (Sec. 3, last
// paragraph) and of the commit of a converged increment.
//
// Spectral layout: S[kz][ky][kx][c], c = 6 tensor components innermost, kx in [0, nx/2]
// (half spectrum of the real-to-complex transform along x), complex values.
// Between iterations S holds the strain with x still in Fourier space and y, z in
// real space ("x-spectral" form).  One iteration:
//   k_xpass   inverse x-FFT -> eps(x) -> per-voxel MC update -> sigma, tau = sigma - C0:eps
//             -> forward x-FFT (out of place); sums of sigma (per thread and in-warp in
//             the field precision, across warps and CTAs in FP64); the last CTA forms
//             <sigma>, the stress-constraint error and the mixed-load update.
//   k_line_pencil / k_line   forward y-FFT (in place)
//   k_zgreen  forward z-FFT -> eps_hat = -Gamma0(kappa):tau_hat / N, eps_hat(0) = E,
//             equilibrium residual (FP64 sums) -> inverse z-FFT (in place)
//   k_line_pencil / k_line   inverse y-FFT (in place)
#pragma once

#include "constitutive.cuh"
#include "fft_reg.cuh"
#include "fft_smem.cuh"
#include "rve_common.cuh"

namespace rve {

// ---------------------------------------------------------------- reductions --------
template <int NV>
__device__ __forceinline__ void warp_sum(double* v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
}

// Fixed-order block sum; result valid in every lane of warp 0.  blockDim % 32 == 0.
template <int NV>
__device__ __forceinline__ void block_sum(double* v, double (*red)[kNumRed]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  warp_sum<NV>(v);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[wid][i] = v[i];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = lane < nw ? red[lane][i] : 0.0;
    warp_sum<NV>(v);
  }
  __syncthreads();
}

// A CTA's place in the (2-D) grid of one RVE's pass: coordinates, linear index and the
// pass's CTA count.  A stand-alone launch takes them from blockIdx / gridDim; a grouped
// launch over several RVEs (k_*_group) from the CTA's slice of the combined grid, so every
// RVE's CTAs compute and reduce exactly as in their own launch.
struct Cta {
  unsigned bx, by, lin, count;
};
__device__ __forceinline__ Cta own_grid() {
  return Cta{blockIdx.x, blockIdx.y, blockIdx.x + gridDim.x * blockIdx.y, gridDim.x * gridDim.y};
}

// Stores this CTA's sums and returns true (in all threads) in the CTA that finished last.
template <int NV>
__device__ __forceinline__ bool publish_partial(double* v, double* partial, unsigned int* counter,
                                                double (*red)[kNumRed], int* s_last, const Cta& cta) {
  block_sum<NV>(v, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) partial[(size_t)cta.lin * kNumRed + i] = v[i];
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    *s_last = (prev == cta.count - 1) ? 1 : 0;
  }
  __syncthreads();
  return *s_last != 0;
}

// publish_partial for NV sums held in the field precision T: the in-warp shuffle tree runs
// in T (in float, the adds of GB300's slow FP64 pipe are kept out of every thread), the
// warp sums are converted and added across warps in FP64.  For T = double this is
// publish_partial's arithmetic.
template <typename T, int NV>
__device__ __forceinline__ bool publish_partial_t(const T* s, double* partial, unsigned int* counter,
                                                  double (*red)[kNumRed], int* s_last, const Cta& cta) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = s[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[wid][i] = (double)v[i];
  __syncthreads();
  if (wid == 0) {
    double w[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) w[i] = lane < nw ? red[lane][i] : 0.0;
    warp_sum<NV>(w);
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < NV; ++i) partial[(size_t)cta.lin * kNumRed + i] = w[i];
      __threadfence();
      const unsigned int prev = atomicAdd(counter, 1u);
      *s_last = (prev == cta.count - 1) ? 1 : 0;
    }
  }
  __syncthreads();
  return *s_last != 0;
}

// Deterministic grand total of all CTAs' partials (fixed assignment and tree order).
template <int NV>
__device__ __forceinline__ void total_partials(const double* partial, double* v, double (*red)[kNumRed],
                                               unsigned int count) {
  __threadfence();
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.0;
  for (int b = threadIdx.x; b < (int)count; b += blockDim.x)
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __ldcg(&partial[(size_t)b * kNumRed + i]);
  block_sum<NV>(v, red);
}

__device__ __forceinline__ double mandel_w(int a) { return a < 3 ? 1.0 : 1.41421356237309504880; }

// ---------------------------------------------------------------- x pass -----------
// The x pass's arguments that do not depend on the grid: material, load, increment and
// the rate-root tables.  RVEs stepped as one group share them (identical material and
// load), so a grouped launch reads them at fixed parameter offsets.
template <typename T>
struct XCommon {
  const T* root_tab;  // rate-root tables: kRootTabs values
  MatDev<T> M;
  LoadDev ld;
  T dt;
  int nsub;
};

template <typename T>
struct XArgs {
  int nx, ny, nz, H, L;
  int xs;  // line stride of the shared-memory x sequences: nx + 1 for the register-split lengths, else nx
  long long nvox;
  FftDim dx;
  const C2<T>* tw;
  const C2<T>* spec_in;
  C2<T>* spec_out;
  T* ep;
  T* v;
  T* al;
  T* eps_n;
  T* sig_n;
  const uint32_t* grain;
  const T* Rg;
  XCommon<T> k;
  const int* done;  // iteration launches return at once when *done != 0 (NULL: always run)
  double* partial;
  unsigned int* counter;
  IterStatus* st;
  int it;  // iteration index; < 0: read it from st->it_dev (graph mode)
  // graph-mode commit: runs only if the increment converged, reading the strain spectrum
  // of the converged iteration it* (cand[0] for it* = 0, cand[1] for odd, cand[2] for even)
  int pick;
  const C2<T>* cand[3];
  // linear-law mode (NP == kLinearLaw, the adjoint solve): s = B eps - g per voxel,
  // B 36 x nvox (entry (r, c) at (r * 6 + c) * nvox + voxel), g 6 x nvox
  const T* lin_B;
  const T* lin_g;
  // one byte per warp's 32 consecutive voxels (index voxel / 32 of its first voxel): 1 when
  // some voxel of the group flowed in the increment's first trial iteration, which then
  // skips the elastic-increment test in the later ones (NULL: always test)
  unsigned char* flow;
};

// The x transforms of a CTA's nseq packed lines (stride xs >= N + 1 in shared memory) for
// a length N = N1 N2 with a register split: step 1 from a into b, step 2 back into a in natural
// order.  Consecutive threads take consecutive lines, so with an odd stride both steps
// are free of bank conflicts.  Contains barriers: every thread of the CTA calls it.
template <typename T, int SIGN, int N1, int N2>
__device__ __forceinline__ void xlines_pencil(C2<T>* a, C2<T>* b, int nseq, int xs, const C2<T>* tw, int tid,
                                              int nthr) {
  for (int w = tid; w < nseq * N1; w += nthr) {
    const int q = w % nseq, n1 = w / nseq;
    C2<T> v[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = a[(size_t)q * xs + n1 + N1 * n2];
    pencil_step1<T, SIGN, N1, N2>(v, n1, b + (size_t)q * xs, tw);
  }
  __syncthreads();
  for (int w = tid; w < nseq * N2; w += nthr) {
    const int q = w % nseq, k2 = w / nseq;
    C2<T> u[N1];
    pencil_step2<T, SIGN, N1, N2>(u, k2, b + (size_t)q * xs);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) a[(size_t)q * xs + k2 + N2 * k1] = u[k1];
  }
  __syncthreads();
}

template <typename T, int SIGN, int N>
__device__ __forceinline__ void xlines_split(C2<T>* a, C2<T>* b, int nseq, int xs, const C2<T>* tw, int tid,
                                             int nthr) {
  xlines_pencil<T, SIGN, PencilSplit<N>::N1, PencilSplit<N>::N2>(a, b, nseq, xs, tw, tid, nthr);
}

// The CTA's x transforms: register two-step transforms for the lengths of the PencilSplit
// table (64, 96, 128, 160, 256; result in a), shared-memory Stockham passes otherwise
// (result in a or b, returned).
template <typename T, int SIGN>
__device__ __forceinline__ C2<T>* xlines_fft(C2<T>* a, C2<T>* b, const FftDim& d, int nseq, int xs, const C2<T>* tw,
                                             int tid, int nthr) {
  switch (d.n) {
    case 64: xlines_split<T, SIGN, 64>(a, b, nseq, xs, tw, tid, nthr); return a;
    case 96: xlines_split<T, SIGN, 96>(a, b, nseq, xs, tw, tid, nthr); return a;
    case 128: xlines_split<T, SIGN, 128>(a, b, nseq, xs, tw, tid, nthr); return a;
    case 160: xlines_split<T, SIGN, 160>(a, b, nseq, xs, tw, tid, nthr); return a;
    case 256: xlines_split<T, SIGN, 256>(a, b, nseq, xs, tw, tid, nthr); return a;
    default: return smem_fft<T, SIGN>(a, b, d, nseq, xs, tw, tid, nthr);
  }
}

constexpr int kXThreads = 128;
// Minimum resident x-pass CTAs per SM requested from the register allocator.  Float: 3
// (at most 168 registers; the constitutive update is latency-bound at 2 CTAs, and 3 run
// 8 % faster on the 128^3 workload despite a few spilled values).  Double: 1.
template <typename T> struct XMinBlocks { static constexpr int value = 1; };
template <> struct XMinBlocks<float> { static constexpr int value = 3; };

// One CTA of the x pass (see the file header) at grid place `cta`; k holds a.k or the
// group's common arguments.
template <typename T, bool COMMIT, int NP>
__device__ __forceinline__ void xpass_cta(const XArgs<T>& a, const XCommon<T>& k, const Cta& cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32][kNumRed];
  __shared__ int s_last;
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* b0 = tw + a.nx;
  C2<T>* b1 = b0 + 3 * a.L * a.xs;
  T* tab = reinterpret_cast<T*>(b1 + 3 * a.L * a.xs);  // kRootTabs
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nx = a.nx, H = a.H, half = nx / 2, xs = a.xs;
  const size_t NL = (size_t)a.ny * a.nz;
  const int line0 = (int)cta.bx * a.L;
  const int nl = min(a.L, (int)(NL - line0));
  if (a.done && *a.done) return;  // increment already decided: speculative launch
  const size_t nvox = (size_t)a.nvox;
  const int it = a.it >= 0 ? a.it : a.st->it_dev;
  const C2<T>* spec_in = a.spec_in;
  if (COMMIT && a.pick) {
    if (a.st->done != 1) return;  // not converged: the host rolls the increment back
    const int k = a.st->done_it;
    spec_in = k == 0 ? a.cand[0] : ((k & 1) ? a.cand[1] : a.cand[2]);
  }

  for (int i = tid; i < nx; i += nthr) tw[i] = a.tw[i];
  if (NP != 0 && NP != kLinearLaw)
    for (int i = tid; i < kRootTabs; i += nthr) tab[i] = k.root_tab[i];
  // pack component pairs (2p, 2p+1) of each line as one complex Hermitian-extended
  // sequence Z = A + iB, so one complex inverse FFT yields both real lines
  // (spectra are component-interleaved: entry (line, kx, c) at (line * H + kx) * 6 + c,
  // so consecutive threads read consecutive component pairs of the CTA's lines)
  for (int w = tid; w < 3 * nl * H; w += nthr) {
    const int p = w % 3;
    const int r = w / 3;
    const int xi = r % H, l = r / H;
    const int q = p * nl + l;
    const size_t e0 = (((size_t)line0 + l) * H + xi) * 6 + 2 * p;
    C2<T> A = spec_in[e0];
    C2<T> B = spec_in[e0 + 1];
    if (xi == 0 || xi == half) {
      A.y = T(0);
      B.y = T(0);
    }
    C2<T>* seq = b0 + (size_t)q * xs;
    seq[xi] = mk<T>(A.x - B.y, A.y + B.x);
    if (xi > 0 && xi < half) seq[nx - xi] = mk<T>(A.x + B.y, B.x - A.y);
  }
  __syncthreads();
  C2<T>* res = xlines_fft<T, +1>(b0, b1, a.dx, 3 * nl, xs, tw, tid, nthr);
  C2<T>* oth = (res == b0) ? b1 : b0;

  double acc[kNumRed];
#pragma unroll
  for (int i = 0; i < kNumRed; ++i) acc[i] = 0.0;
  // the thread's stresses are summed in the field precision over its few voxels (4 at
  // most in float) and added to the FP64 block sum once
  T sacc[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  for (int t = tid; t < nl * nx; t += nthr) {
    const int l = t / nx, x = t - l * nx;
    const size_t vox = ((size_t)line0 + l) * nx + x;
    T eps[6], epsn[6], sig[6], R[9];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const C2<T> z = res[(size_t)(p * nl + l) * xs + x];
      eps[2 * p] = z.x;
      eps[2 * p + 1] = z.y;
    }
    if constexpr (NP == kLinearLaw) {
      (void)epsn;
      (void)R;
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        T sr = -a.lin_g[r * nvox + vox];
#pragma unroll
        for (int c = 0; c < 6; ++c) sr += a.lin_B[(r * 6 + c) * nvox + vox] * eps[c];
        sig[r] = sr;
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) acc[c] += (double)sig[c];
      if (COMMIT) {
#pragma unroll
        for (int c = 0; c < 6; ++c) a.eps_n[c * nvox + vox] = eps[c];
        continue;
      }
    } else {
  #pragma unroll
      for (int c = 0; c < 6; ++c) epsn[c] = a.eps_n[c * nvox + vox];
      MPState<T> y;
  #pragma unroll
      for (int c = 0; c < 6; ++c) y.ep[c] = a.ep[c * nvox + vox];
  #pragma unroll
      for (int c = 0; c < 16; ++c) y.v[c] = a.v[c * nvox + vox];
  #pragma unroll
      for (int c = 0; c < 12; ++c) y.al[c] = a.al[c * nvox + vox];
      const uint32_t g = a.grain[vox];
  #pragma unroll
      for (int i = 0; i < 9; ++i) R[i] = a.Rg[(size_t)g * 9 + i];
      // The elastic-increment test saves work only where all 32 voxels of a warp stay
      // elastic; in the developed plastic regime it is wasted.  Iteration 0 of an increment
      // (and the commit) always tests and records per warp whether any voxel flowed;
      // warps that flowed skip the test in the increment's later iterations.
      const size_t grp = ((size_t)line0 * nx + (size_t)(t - (tid & 31))) >> 5;
      const bool record = !COMMIT && a.flow != nullptr && it == 0;
      const bool check = COMMIT || a.flow == nullptr || it == 0 || a.flow[grp] == 0;
      const bool flowed = mc_voxel<T, NP>(k.M, R, epsn, eps, y, k.dt, k.nsub, sig, tab, check);
      if (record) {
        const bool any = __any_sync(__activemask(), flowed);
        if ((tid & 31) == 0) a.flow[grp] = any ? 1 : 0;
      }
  #pragma unroll
      for (int c = 0; c < 6; ++c) sacc[c] += sig[c];
      if (COMMIT) {
  #pragma unroll
        for (int c = 0; c < 6; ++c) a.ep[c * nvox + vox] = y.ep[c];
  #pragma unroll
        for (int c = 0; c < 16; ++c) a.v[c * nvox + vox] = y.v[c];
  #pragma unroll
        for (int c = 0; c < 12; ++c) a.al[c * nvox + vox] = y.al[c];
  #pragma unroll
        for (int c = 0; c < 6; ++c) {
          a.eps_n[c * nvox + vox] = eps[c];
          a.sig_n[c * nvox + vox] = sig[c];
        }
        acc[6] += (double)von_mises6<T>(sig);
        acc[7] += 1.41421356237309504880 * ((double)y.v[12] + (double)y.v[13] + (double)y.v[14] + (double)y.v[15]);
        double vs = 0.0;
  #pragma unroll
        for (int c = 0; c < 12; ++c) vs += (double)y.v[c];
        acc[8] += vs;
        continue;
      }
    }
    {
      const T tr = k.M.lam0 * (eps[0] + eps[1] + eps[2]);
      const T m2 = T(2) * k.M.mu0;
      T tau[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) tau[c] = sig[c] - m2 * eps[c] - (c < 3 ? tr : T(0));
#pragma unroll
      for (int p = 0; p < 3; ++p) res[(size_t)(p * nl + l) * xs + x] = mk<T>(tau[2 * p], tau[2 * p + 1]);
    }
  }
  if constexpr (COMMIT || NP == kLinearLaw) {
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += (double)sacc[c];
  }
  if (!COMMIT) {
    __syncthreads();
    C2<T>* out = xlines_fft<T, -1>(res, oth, a.dx, 3 * nl, xs, tw, tid, nthr);
    // unpack: A = (Z_k + conj Z_{n-k}) / 2, B = (Z_k - conj Z_{n-k}) / (2i)
    for (int w = tid; w < 3 * nl * H; w += nthr) {
      const int p = w % 3;
      const int r = w / 3;
      const int xi = r % H, l = r / H;
      const int q = p * nl + l;
      const C2<T> Z = out[(size_t)q * xs + xi];
      const C2<T> Zm = out[(size_t)q * xs + (xi == 0 ? 0 : nx - xi)];
      const C2<T> A = mk<T>(T(0.5) * (Z.x + Zm.x), T(0.5) * (Z.y - Zm.y));
      const C2<T> B = mk<T>(T(0.5) * (Z.y + Zm.y), T(-0.5) * (Z.x - Zm.x));
      const size_t e0 = (((size_t)line0 + l) * H + xi) * 6 + 2 * p;
      a.spec_out[e0] = A;
      a.spec_out[e0 + 1] = B;
    }
  }
  // trial iterations sum the 6 stress components (in-warp in the field precision); the
  // commit and the linear-law mode all slots in FP64
  constexpr bool kSix = !COMMIT && NP != kLinearLaw;
  bool last;
  if constexpr (kSix) last = publish_partial_t<T, 6>(sacc, a.partial, a.counter, red, &s_last, cta);
  else last = publish_partial<kNumRed>(acc, a.partial, a.counter, red, &s_last, cta);
  if (last) {
    if constexpr (kSix) total_partials<6>(a.partial, acc, red, cta.count);
    else total_partials<kNumRed>(a.partial, acc, red, cta.count);
    if (tid == 0) {
      IterStatus* st = a.st;
      const double inv = 1.0 / (double)a.nvox;
      double S[6];
      int bad = 0;
      for (int c = 0; c < 6; ++c) {
        S[c] = acc[c] * inv;
        st->sig_mean[c] = S[c];
        bad |= !isfinite(S[c]);
      }
      if (COMMIT) {
        st->eff[0] = acc[6] * inv;
        st->eff[1] = acc[7] * inv * 0.25;
        st->eff[2] = acc[8] * inv / 12.0;
        bad |= !isfinite(acc[6]) | !isfinite(acc[7]) | !isfinite(acc[8]);
      } else {
        // mixed-load update of the free components (Mandel form)
        const LoadDev& ld = k.ld;
        double miss[6], nm = 0.0, ns = 0.0;
        for (int c = 0; c < 6; ++c) {
          const double sm = S[c] * mandel_w(c);
          miss[c] = ld.free_mask[c] ? sm - ld.Sigma_m[c] : 0.0;
          nm += miss[c] * miss[c];
          ns += sm * sm;
        }
        st->cF = ld.any_free ? sqrt(nm) / fmax(sqrt(ns), ld.s_ref) : 0.0;
        const double* Ec = st->E[it & 1];
        double* En = st->E[(it + 1) & 1];
        for (int c = 0; c < 6; ++c) {
          double em = Ec[c] * mandel_w(c);
          if (ld.free_mask[c]) {
            double corr = 0.0;
            for (int b = 0; b < 6; ++b) corr += ld.Minv[c * 6 + b] * miss[b];
            em -= corr;
          }
          En[c] = em / mandel_w(c);
        }
      }
      st->nan_flag |= bad ? (COMMIT ? 4 : 1) : 0;
      *a.counter = 0u;
    }
  }
}

template <typename T, bool COMMIT, int NP>
__global__ void __launch_bounds__(kXThreads, XMinBlocks<T>::value) k_xpass(const XArgs<T> a) {
  xpass_cta<T, COMMIT, NP>(a, a.k, own_grid());
}

// ---------------------------------------------------------------- line FFT pass -----
// Transforms, in place, lines of length d.n along an axis with element stride `stride`
// (complex units), for NC components at once.  Element (line j, kx offset hh, component
// c) of the CTA at grid place (bx, o = by) sits at
//   (o / n_o2) * A + (o % n_o2) * B + (h0 + hh) * hstride + c + j * stride,
// h0 = bx * HC.  The solver's spectra are component-interleaved (NC = 6,
// hstride = 6: each (j, kx chunk) row is HC * 6 contiguous values); the stand-alone FFT
// entry points use component-major spectra (NC = 1, hstride = 1).
template <typename T>
struct LineArgs {
  FftDim d;
  const C2<T>* tw;
  C2<T>* spec;
  int H, HC, n_o2, NC, hstride;
  const int* done;  // as in XArgs
  long long stride, A, B;
};

// Moves a tile between global memory and shared-memory FFT sequences.  Global: n rows of
// `row` contiguous complex values, row j at g + j * gstride.  Shared: value r of row j at
// s[q(r) * ps + j], q(r) = (r % NC) * hc + r / NC (component-interleaved rows become one
// sequence per component and kx).  Each thread keeps one column (or, in float with an even
// row, a 16-byte pair of columns) and walks the rows, so the loop carries no divisions and
// several loads are in flight.  Returns without a barrier.
template <typename T, bool LOAD>
__device__ __forceinline__ void tile_move(C2<T>* s, int ps, C2<T>* g, size_t gstride, int n, int row, int NC, int hc,
                                          int tid, int nthr) {
  constexpr bool kPairable = sizeof(C2<T>) == 8;
  if (kPairable && (row % 2) == 0 && (reinterpret_cast<size_t>(g) % 16) == 0 && (gstride % 2) == 0) {
    const int rp = row / 2;
    const int R = nthr / rp;
    if (tid >= R * rp) return;
    const int r = 2 * (tid % rp), j0 = tid / rp;
    C2<T>* s0 = s + (size_t)((r % NC) * hc + r / NC) * ps;
    C2<T>* s1 = s + (size_t)(((r + 1) % NC) * hc + (r + 1) / NC) * ps;
    float4* gv = reinterpret_cast<float4*>(g + r);
    const size_t vstride = gstride / 2;
#pragma unroll 4
    for (int j = j0; j < n; j += R) {
      if (LOAD) {
        const float4 v = gv[(size_t)j * vstride];
        s0[j] = mk<T>(T(v.x), T(v.y));
        s1[j] = mk<T>(T(v.z), T(v.w));
      } else {
        const C2<T> a0 = s0[j], a1 = s1[j];
        gv[(size_t)j * vstride] = make_float4(float(a0.x), float(a0.y), float(a1.x), float(a1.y));
      }
    }
    return;
  }
  const int R = nthr / row;
  if (tid >= R * row) return;
  const int r = tid % row, j0 = tid / row;
  C2<T>* sq = s + (size_t)((r % NC) * hc + r / NC) * ps;
  C2<T>* gr = g + r;
#pragma unroll 4
  for (int j = j0; j < n; j += R) {
    if (LOAD) sq[j] = gr[(size_t)j * gstride];
    else gr[(size_t)j * gstride] = sq[j];
  }
}

constexpr int kLineThreads = 256;

template <typename T, int SIGN>
__device__ __forceinline__ void line_cta(const LineArgs<T>& a, const Cta& cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  const int n = a.d.n;
  const int ps = n + 1;  // padded sequence stride
  const int NC = a.NC;
  C2<T>* b0 = tw + n;
  C2<T>* b1 = b0 + (size_t)NC * a.HC * ps;
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (a.done && *a.done) return;
  const int h0 = (int)cta.bx * a.HC;
  const int hc = min(a.HC, a.H - h0);
  const int o = (int)cta.by;
  const size_t base = (size_t)(o / a.n_o2) * a.A + (size_t)(o % a.n_o2) * a.B + (size_t)h0 * a.hstride;
  const int row = hc * NC;  // values per line position, contiguous when hstride == NC
  for (int i = tid; i < n; i += nthr) tw[i] = a.tw[i];
  if (a.hstride == NC) {  // the row's values are contiguous
    tile_move<T, true>(b0, ps, a.spec + base, (size_t)a.stride, n, row, NC, hc, tid, nthr);
  } else {
    for (int w = tid; w < row * n; w += nthr) {
      const int rc = w % row, j = w / row;
      const int c = rc % NC, hh = rc / NC;
      b0[(size_t)(c * hc + hh) * ps + j] = a.spec[base + (size_t)j * a.stride + (size_t)hh * a.hstride + c];
    }
  }
  __syncthreads();
  C2<T>* res = smem_fft<T, SIGN>(b0, b1, a.d, row, ps, tw, tid, nthr);
  if (a.hstride == NC) {
    tile_move<T, false>(res, ps, a.spec + base, (size_t)a.stride, n, row, NC, hc, tid, nthr);
  } else {
    for (int w = tid; w < row * n; w += nthr) {
      const int rc = w % row, j = w / row;
      const int c = rc % NC, hh = rc / NC;
      a.spec[base + (size_t)j * a.stride + (size_t)hh * a.hstride + c] = res[(size_t)(c * hc + hh) * ps + j];
    }
  }
}

template <typename T, int SIGN>
__global__ void __launch_bounds__(kLineThreads) k_line(const LineArgs<T> a) {
  line_cta<T, SIGN>(a, own_grid());
}

// The y pass for a line length N = N1 N2 with a register split (fft_reg.cuh), on the solver's
// component-interleaved spectra (NC = hstride = 6).  CTA (kx chunk, outer index) as in
// k_line; its S = 6 hc lines s sit contiguously in every row.  Thread t = n1 SP + s
// (SP = 6 HC) loads column n1 of line s straight from global memory (rows n1 + N1 n2),
// transforms it in registers and parks it in shared memory; then each column k2 of a line
// is transformed and written back to rows k2 + N2 k1.  One barrier between the steps.
constexpr int kPencilThreads = 384;  // at most N1 * NC * HC threads per CTA

// NC = 6 serves the solver's component-interleaved spectra; NC = 1 (hstride 1) the
// stand-alone transforms' component-major spectra, one component per CTA.
template <typename T, int SIGN, int N1, int N2, int NC = 6>
__device__ __forceinline__ void line_pencil_cta(const LineArgs<T>& a, const Cta& cta) {
  constexpr int N = N1 * N2;
  constexpr int ps = N + 1;  // padded line stride in shared memory
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* buf = tw + N;
  if (a.done && *a.done) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int SP = NC * a.HC;
  const int h0 = (int)cta.bx * a.HC;
  const int S = NC * min(a.HC, a.H - h0);
  const int o = (int)cta.by;
  C2<T>* g = a.spec + (size_t)(o / a.n_o2) * a.A + (size_t)(o % a.n_o2) * a.B + (size_t)h0 * NC;
  const size_t gs = (size_t)a.stride;
  const int s = tid % SP, n1 = tid / SP;
  const bool mine = s < S && n1 < N1;  // the CTA has N1 * SP threads rounded up to warps
  C2<T> v[N2];
  if (mine) {
#pragma unroll
    for (int q = 0; q < N2; ++q) v[q] = g[(size_t)(n1 + N1 * q) * gs + s];
  }
  for (int i = tid; i < N; i += nthr) tw[i] = a.tw[i];
  __syncthreads();
  if (mine) pencil_step1<T, SIGN, N1, N2>(v, n1, buf + (size_t)s * ps, tw);
  __syncthreads();
  for (int col = tid; col < N2 * SP; col += nthr) {
    const int s2 = col % SP, k2 = col / SP;
    if (s2 < S) {
      C2<T> w[N1];
      pencil_step2<T, SIGN, N1, N2>(w, k2, buf + (size_t)s2 * ps);
#pragma unroll
      for (int q = 0; q < N1; ++q) g[(size_t)(k2 + N2 * q) * gs + s2] = w[q];
    }
  }
}

template <typename T, int SIGN, int N1, int N2, int NC>
__global__ void __launch_bounds__(kPencilThreads) k_line_pencil(const LineArgs<T> a) {
  line_pencil_cta<T, SIGN, N1, N2, NC>(a, own_grid());
}

// ---------------------------------------------------------------- z pass + Green ----
template <typename T>
struct ZArgs {
  int nx, ny, nz, H, HC;
  long long nvox;
  FftDim dz;
  const C2<T>* tw;
  C2<T>* spec;
  const C2<T>* P_prev;
  C2<T>* P_out;
  const T* kx;  // per dimension, 2*N values: Willot (sin, cos) of pi xi/N, or MS (freq, 0)
  const T* ky;
  const T* kzt;
  int scheme;   // 0 Willot, 1 Moulinec-Suquet
  ConvDev conv;
  const int* done;
  T lam0, mu0, invN;
  double* partial;
  unsigned int* counter;
  IterStatus* st;
  int it;  // iteration index; < 0: read it from st->it_dev and advance it (graph mode)
  int has_cond;  // graph mode: clear the loop condition once the increment is decided
  cudaGraphConditionalHandle cond;
};

constexpr int kZThreads = 256;

// The six components of a spectral point, contiguous at p: 16-byte vector accesses when
// vec (both tau_hat spectra 16-byte aligned; every point's offset 6 * 8 or 6 * 16 bytes
// keeps that alignment), else one complex value at a time.
template <typename T>
__device__ __forceinline__ void load_point6(const C2<T>* p, C2<T>* v, bool vec) {
  if constexpr (sizeof(C2<T>) == 8) {
    if (vec) {
      const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float4 f = q[i];
        v[2 * i] = mk<T>(f.x, f.y);
        v[2 * i + 1] = mk<T>(f.z, f.w);
      }
      return;
    }
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) v[c] = p[c];
}
template <typename T>
__device__ __forceinline__ void store_point6(C2<T>* p, const C2<T>* v, bool vec) {
  if constexpr (sizeof(C2<T>) == 8) {
    if (vec) {
      float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
      for (int i = 0; i < 3; ++i) q[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
      return;
    }
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) p[c] = v[c];
}

// Green operator step of one spectral point (kx index h, ky index j, kz): t holds tau_hat
// on entry and the new strain spectrum on exit; tau_hat is kept for the next iteration's
// residual (P_out) and the point's weighted residual term |kappa . sigma_hat|^2 is returned.
template <typename T>
__device__ __forceinline__ T green_point(const ZArgs<T>& a, int h, int j, int kz, const double* En, T coef,
                                         bool vec, C2<T>* t) {
  T k0, k1, k2;
  if (a.scheme == 0) {
    const T sx = a.kx[2 * h], cx = a.kx[2 * h + 1];
    const T sy = a.ky[2 * j], cy = a.ky[2 * j + 1];
    const T sz = a.kzt[2 * kz], cz = a.kzt[2 * kz + 1];
    k0 = sx * cy * cz;
    k1 = cx * sy * cz;
    k2 = cx * cy * sz;
  } else {
    k0 = a.kx[2 * h];
    k1 = a.ky[2 * j];
    k2 = a.kzt[2 * kz];
  }
  const size_t g0 = (((size_t)kz * a.ny + j) * a.H + h) * 6;
  T rterm;
  // equilibrium residual kappa . sigma_hat = kappa . (tau_hat - tau_hat_prev)
  {
    C2<T> d[6];
    load_point6<T>(a.P_prev + g0, d, vec);
    store_point6<T>(a.P_out + g0, t, vec);
#pragma unroll
    for (int c = 0; c < 6; ++c) d[c] = csub<T>(t[c], d[c]);
    // symmetric order (11,22,33,23,13,12): row i of d times kappa.  The point's term and
    // its column's sum over kz are formed in the field precision (relative rounding
    // below 1e-5 in float, on an error compared with tolerances of 1e-6 and above); the
    // sum over columns is FP64.
    const T r0x = d[0].x * k0 + d[5].x * k1 + d[4].x * k2;
    const T r0y = d[0].y * k0 + d[5].y * k1 + d[4].y * k2;
    const T r1x = d[5].x * k0 + d[1].x * k1 + d[3].x * k2;
    const T r1y = d[5].y * k0 + d[1].y * k1 + d[3].y * k2;
    const T r2x = d[4].x * k0 + d[3].x * k1 + d[2].x * k2;
    const T r2y = d[4].y * k0 + d[3].y * k1 + d[2].y * k2;
    const T wgt = (h == 0 || 2 * h == a.nx) ? T(1) : T(2);
    rterm = wgt * (r0x * r0x + r0y * r0y + r1x * r1x + r1y * r1y + r2x * r2x + r2y * r2y);
  }
  const T kk = k0 * k0 + k1 * k1 + k2 * k2;
  if (h == 0 && j == 0 && kz == 0) {
#pragma unroll
    for (int c = 0; c < 6; ++c) t[c] = mk<T>(T(En[c]), T(0));
  } else if (!(kk > T(0))) {
#pragma unroll
    for (int c = 0; c < 6; ++c) t[c] = mk<T>(T(0), T(0));
  } else {
    // Gamma0 is homogeneous of degree 0 in kappa: with the unit direction n = kappa/|kappa|,
    // eps_hat = -[ (n_i u_j + n_j u_i) / (2 mu0) - coef n_i n_j (n.u) ] / N,  u = tau_hat n
    const T inv_k = T(1) / sqrt(kk);
    const T n0 = k0 * inv_k, n1 = k1 * inv_k, n2 = k2 * inv_k;
    const C2<T> u0 = mk<T>(t[0].x * n0 + t[5].x * n1 + t[4].x * n2, t[0].y * n0 + t[5].y * n1 + t[4].y * n2);
    const C2<T> u1 = mk<T>(t[5].x * n0 + t[1].x * n1 + t[3].x * n2, t[5].y * n0 + t[1].y * n1 + t[3].y * n2);
    const C2<T> u2 = mk<T>(t[4].x * n0 + t[3].x * n1 + t[2].x * n2, t[4].y * n0 + t[3].y * n1 + t[2].y * n2);
    const C2<T> nun = mk<T>(n0 * u0.x + n1 * u1.x + n2 * u2.x, n0 * u0.y + n1 * u1.y + n2 * u2.y);
    const T ia = -a.invN / (T(2) * a.mu0);
    const T ib = a.invN * coef;
    const T nv[3] = {n0, n1, n2};
    const C2<T> uv[3] = {u0, u1, u2};
    const int ii[6] = {0, 1, 2, 1, 0, 0};
    const int jj[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const T ni = nv[ii[c]], nj = nv[jj[c]];
      const C2<T> ui = uv[ii[c]], uj = uv[jj[c]];
      const T nij = ni * nj;
      t[c] = mk<T>(ia * (ni * uj.x + nj * ui.x) + ib * nij * nun.x, ia * (ni * uj.y + nj * ui.y) + ib * nij * nun.y);
    }
  }
  return rterm;
}

// The second step of the two-step transform on every column of the CTA's lines, in place:
// the column k2 of line s (slots k2 N1 + n1, n1 = 0 .. N1 - 1) is replaced by its N1-point
// DFT, each thread reading and writing only its own columns' slots.  Forward (SIGN < 0):
// slot k2 N1 + k1 then holds X[k2 + N2 k1].  Inverse (SIGN > 0, the first step of the
// transposed inverse): the slots hold X[k2 + N2 k1] on entry and
// Z[n1][k2] = W^(n1 k2) sum_k1 X[k2 + N2 k1] W_N1^(n1 k1) at slot k2 N1 + n1 on exit,
// W = e^(2 pi i / N), W_N1 = e^(2 pi i / N1) (tw[e] = e^(-2 pi i e / N)).
template <typename T, int SIGN, int N1, int N2>
__device__ __forceinline__ void pencil_cols_inplace(C2<T>* b, int ps, int SP, int S, const C2<T>* tw, int tid,
                                                    int nthr) {
  constexpr int kCols = (N2 + N1 - 1) / N1;  // columns per thread (N2 * SP columns, >= N1 * SP threads)
#pragma unroll
  for (int r = 0; r < kCols; ++r) {
    const int col = tid + r * nthr;
    const int s2 = col % SP, k2 = col / SP;
    if (col < N2 * SP && s2 < S) {
      C2<T>* line = b + (size_t)s2 * ps;
      C2<T> w[N1];
      pencil_step2<T, SIGN, N1, N2>(w, k2, line);
      if constexpr (SIGN > 0) {
#pragma unroll
        for (int q = 1; q < N1; ++q)
          if (k2 > 0) w[q] = cmulc<T>(w[q], tw[q * k2]);
      }
#pragma unroll
      for (int q = 0; q < N1; ++q) line[k2 * N1 + q] = w[q];
    }
  }
}

// N1 = N2 = 0: Stockham transforms of any supported nz in shared memory (two buffers,
// line of component c and chunk column hh at (c hc + hh) ps); N1 N2 = nz: the two-step
// register transforms of fft_reg.cuh (one buffer, line s = 6 hh + c at s ps, as in the
// global rows).  The register path runs the forward transform's second step in place, so
// the Green step reads the spectrum in that step's slot order (point kz = k2 + N2 k1 at
// slot k2 N1 + k1), and the inverse as the transposed two-step transform (the N1-point
// DFTs of the columns first, in place, then the N2-point DFTs straight to global memory):
// three barriers between the global load and the global store; twiddles are read through
// L1.
template <typename T, int N1, int N2>
__device__ __forceinline__ void zgreen_cta(const ZArgs<T>& a, const Cta& cta, double (*red)[kNumRed], int& s_last) {
  constexpr bool kPencil = N1 > 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nz = a.nz;
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  const int ps = nz + 1;  // padded sequence stride
  C2<T>* b0 = tw + nz;
  C2<T>* b1 = b0 + (size_t)6 * a.HC * ps;
  T* cres = reinterpret_cast<T*>((kPencil ? b0 : b1) + (size_t)6 * a.HC * ps);  // HC * nz residual terms
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (a.done && *a.done) return;
  const int j = (int)cta.by;
  const int h0 = (int)cta.bx * a.HC;
  const int hc = min(a.HC, a.H - h0);
  const size_t H = a.H, ny = a.ny;
  C2<T>* gz = a.spec + ((size_t)j * H + h0) * 6;
  const size_t gs = ny * H * 6;
  const bool vec = ((reinterpret_cast<uintptr_t>(a.P_prev) | reinterpret_cast<uintptr_t>(a.P_out)) & 15) == 0;
  const int it = a.it >= 0 ? a.it : a.st->it_dev;
  const double* En = a.st->E[(it + 1) & 1];
  const T coef = (a.lam0 + a.mu0) / (a.mu0 * (a.lam0 + T(2) * a.mu0));
  if constexpr (kPencil) {
    const C2<T>* twg = a.tw;  // e^(-2 pi i e / nz), e < nz (read through L1)
    const int SP = 6 * a.HC, S = 6 * hc;
    const int s = tid % SP, n1 = tid / SP;
    const bool mine = s < S && n1 < N1;  // the CTA has N1 * SP threads rounded up to warps
    // forward z transform: first step from the global rows n1 + N1 n2, second step in place
    if (mine) {
      C2<T> v[N2];
#pragma unroll
      for (int q = 0; q < N2; ++q) v[q] = gz[(size_t)(n1 + N1 * q) * gs + s];
      pencil_step1<T, -1, N1, N2>(v, n1, b0 + (size_t)s * ps, twg);
    }
    __syncthreads();
    pencil_cols_inplace<T, -1, N1, N2>(b0, ps, SP, S, twg, tid, nthr);
    __syncthreads();
    // Green step per point, in slot order (consecutive threads on consecutive slots of
    // the chunk's columns)
    for (int w = tid; w < hc * nz; w += nthr) {
      const int hh = w % hc, sl = w / hc;
      const int kz = sl / N1 + N2 * (sl % N1);
      C2<T> t[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) t[c] = b0[(size_t)(hh * 6 + c) * ps + sl];
      cres[hh * nz + kz] = green_point<T>(a, h0 + hh, j, kz, En, coef, vec, t);
#pragma unroll
      for (int c = 0; c < 6; ++c) b0[(size_t)(hh * 6 + c) * ps + sl] = t[c];
    }
    __syncthreads();
    // inverse z transform: the columns' N1-point DFTs in place, then each thread's
    // N2-point DFT of its column n1 over k2, written to the global rows n1 + N1 n2
    pencil_cols_inplace<T, +1, N1, N2>(b0, ps, SP, S, twg, tid, nthr);
    __syncthreads();
    if (mine) {
      const C2<T>* line = b0 + (size_t)s * ps;
      C2<T> v[N2];
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) v[k2] = line[k2 * N1 + n1];
      dft_reg<T, +1, N2>(v);
#pragma unroll
      for (int q = 0; q < N2; ++q) gz[(size_t)(n1 + N1 * q) * gs + s] = v[q];
    }
  } else {
    for (int i = tid; i < nz; i += nthr) tw[i] = a.tw[i];
    // component-interleaved spectra: for each kz the CTA's hc * 6 values are contiguous
    tile_move<T, true>(b0, ps, gz, gs, nz, 6 * hc, 6, hc, tid, nthr);
    __syncthreads();
    C2<T>* res = smem_fft<T, -1>(b0, b1, a.dz, 6 * hc, ps, tw, tid, nthr);
    C2<T>* oth = (res == b0) ? b1 : b0;
    for (int w = tid; w < hc * nz; w += nthr) {
      const int hh = w % hc, kz = w / hc;
      C2<T> t[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) t[c] = res[(size_t)(c * hc + hh) * ps + kz];
      cres[hh * nz + kz] = green_point<T>(a, h0 + hh, j, kz, En, coef, vec, t);
#pragma unroll
      for (int c = 0; c < 6; ++c) res[(size_t)(c * hc + hh) * ps + kz] = t[c];
    }
    __syncthreads();
    C2<T>* out = smem_fft<T, +1>(res, oth, a.dz, 6 * hc, ps, tw, tid, nthr);
    tile_move<T, false>(out, ps, gz, gs, nz, 6 * hc, 6, hc, tid, nthr);
  }
  // residual: one partial per (ky, kx) column, summed over kz in a fixed order (lane l
  // takes kz = l, l + 32, ...; then a fixed shuffle tree), so the total does not depend on
  // how many kx columns a CTA holds
  {
    const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    for (int hh = wid; hh < hc; hh += nw) {
      T cv = T(0);
      for (int kz = lane; kz < nz; kz += 32) cv += cres[hh * nz + kz];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) cv += __shfl_xor_sync(0xffffffffu, cv, off);
      if (lane == 0) {
        a.partial[(size_t)j * H + h0 + hh] = (double)cv;
        __threadfence();
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(a.counter, 1u);
    s_last = (prev == cta.count - 1) ? 1 : 0;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    // the column partials summed in the order of 256 lanes (8 warps) whatever the block
    // size: lane vl takes b = vl, vl + 256, ... with four accumulators, each warp of lanes
    // adds by a shuffle tree, then warp 0 adds the 8 warp sums
    constexpr int kVL = 256;
    const size_t np = ny * H;
    const int lane = tid & 31;
    for (int vl = tid; vl < kVL; vl += nthr) {
      double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
      size_t b = vl;
      for (; b + 3 * (size_t)kVL < np; b += 4 * (size_t)kVL) {
        q0 += __ldcg(&a.partial[b]);
        q1 += __ldcg(&a.partial[b + kVL]);
        q2 += __ldcg(&a.partial[b + 2 * (size_t)kVL]);
        q3 += __ldcg(&a.partial[b + 3 * (size_t)kVL]);
      }
      for (; b < np; b += kVL) q0 += __ldcg(&a.partial[b]);
      double w = (q0 + q1) + (q2 + q3);
      warp_sum<1>(&w);
      if (lane == 0) red[vl >> 5][0] = w;
    }
    __syncthreads();
    double v[kNumRed];
#pragma unroll
    for (int i = 0; i < kNumRed; ++i) v[i] = 0.0;
    if (tid < 32) {
      v[0] = lane < kVL / 32 ? red[lane][0] : 0.0;
      warp_sum<1>(v);
    }
    if (tid == 0) {
      IterStatus* st = a.st;
      const double* S = st->sig_mean;
      const double nrm =
          fmax(sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2] + 2.0 * (S[3] * S[3] + S[4] * S[4] + S[5] * S[5])),
               a.conv.s_ref);
      st->res_sum = v[0];
      st->e_eq = nrm > 0.0 ? sqrt(v[0]) / ((double)a.nvox * nrm) : 0.0;
      st->nan_flag |= !isfinite(v[0]) ? 2 : 0;
      // convergence decision (equilibrium and stress-constraint errors of iteration it)
      const ConvDev& cv = a.conv;
      cv.hist[2 * it] = st->e_eq;
      cv.hist[2 * it + 1] = st->cF;
      int code = 0;
      if (st->nan_flag) code = 2;
      else if (cv.fixed_iters > 0 ? it + 1 >= cv.fixed_iters : (st->e_eq < cv.tol && st->cF < cv.tol)) code = 1;
      else if (it + 1 >= cv.max_iter) code = 3;
      if (code) {
        st->done_it = it;
        st->done = code;
      }
      if (a.it < 0) st->it_dev = it + 1;
      if (code && a.has_cond) cudaGraphSetConditional(a.cond, 0u);
      *a.counter = 0u;
    }
  }
}

// Resident CTAs per SM the float z pass is compiled for (register cap; its shared memory
// fits as many); double keeps the compiler's choice.
template <typename T, int N1>
struct ZMinBlocks {
  static constexpr int value = sizeof(T) == 4 ? (N1 > 0 ? 3 : 4) : 1;
};

template <typename T, int N1, int N2>
__global__ void __launch_bounds__(N1 > 0 ? kPencilThreads : kZThreads, ZMinBlocks<T, N1>::value)
    k_zgreen(const ZArgs<T> a) {
  __shared__ double red[32][kNumRed];
  __shared__ int s_last;
  zgreen_cta<T, N1, N2>(a, own_grid(), red, s_last);
}

// Graph mode: second bound on the device-side iteration loop, independent of the
// residual kernel's decision: after `limit` executions of the loop body (two iterations
// each) the loop condition is cleared.
template <typename T>
__global__ void k_loop_guard(IterStatus* st, int limit, cudaGraphConditionalHandle cond) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int g = ++st->guard;
    if (g >= limit || st->done) cudaGraphSetConditional(cond, 0u);
  }
}

// ---------------------------------------------------------------- grouped passes ----
// One launch of a pass over several RVEs (an ensemble stepped together): the combined grid
// is the members' own grids laid end to end -- member m owns CTAs start[m] .. start[m+1]-1,
// its grid gx[m] CTAs wide -- and each CTA runs its member's pass exactly as the member's
// own launch would (same arguments, grid place, reductions and decisions), so results are
// those of stepping each RVE alone.  A member whose increment is decided returns at once.
constexpr int kMaxGroup = 16;

// The CTA's member and its place in that member's grid.
__device__ __forceinline__ Cta group_place(const int* start, const int* gx, int n, int* member) {
  int m = 0;
  while (m + 1 < n && (int)blockIdx.x >= start[m + 1]) ++m;
  const unsigned loc = blockIdx.x - (unsigned)start[m];
  *member = m;
  return Cta{loc % (unsigned)gx[m], loc / (unsigned)gx[m], loc, (unsigned)(start[m + 1] - start[m])};
}

template <typename T>
struct XGroup {
  XCommon<T> k;  // shared by every member (the members' own k are not read)
  XArgs<T> m[kMaxGroup];
  int start[kMaxGroup + 1];
  int gx[kMaxGroup];
  int n;
};
template <typename T>
struct LineGroup {
  LineArgs<T> m[kMaxGroup];
  int start[kMaxGroup + 1];
  int gx[kMaxGroup];
  int n;
};
template <typename T>
struct ZGroup {
  ZArgs<T> m[kMaxGroup];
  int start[kMaxGroup + 1];
  int gx[kMaxGroup];
  int n;
};

// the grouped argument blocks are passed by value: within the 32764-byte kernel-parameter limit
static_assert(sizeof(XGroup<double>) <= 32764 && sizeof(LineGroup<double>) <= 32764 &&
                  sizeof(ZGroup<double>) <= 32764,
              "grouped pass arguments exceed the kernel parameter limit");

template <typename T, bool COMMIT, int NP>
__global__ void __launch_bounds__(kXThreads, XMinBlocks<T>::value) k_xpass_group(const __grid_constant__ XGroup<T> g) {
  int m;
  const Cta cta = group_place(g.start, g.gx, g.n, &m);
  xpass_cta<T, COMMIT, NP>(g.m[m], g.k, cta);
}

// y pass of every member: the two-step register transform where the member's length has a
// split and its chunk fits (as launch_line chooses), the Stockham kernel's CTA otherwise.
template <typename T, int SIGN>
__global__ void __launch_bounds__(kPencilThreads) k_line_group(const __grid_constant__ LineGroup<T> g) {
  int m;
  const Cta cta = group_place(g.start, g.gx, g.n, &m);
  const LineArgs<T>& a = g.m[m];
  const bool split = a.NC == 6 && a.hstride == 6 && a.HC <= pencil_max_hc(a.d.n);
  switch (split ? a.d.n : 0) {
    case 64: line_pencil_cta<T, SIGN, PencilSplit<64>::N1, PencilSplit<64>::N2>(a, cta); return;
    case 96: line_pencil_cta<T, SIGN, PencilSplit<96>::N1, PencilSplit<96>::N2>(a, cta); return;
    case 128: line_pencil_cta<T, SIGN, PencilSplit<128>::N1, PencilSplit<128>::N2>(a, cta); return;
    case 160: line_pencil_cta<T, SIGN, PencilSplit<160>::N1, PencilSplit<160>::N2>(a, cta); return;
    case 256: line_pencil_cta<T, SIGN, PencilSplit<256>::N1, PencilSplit<256>::N2>(a, cta); return;
    default: line_cta<T, SIGN>(a, cta); return;
  }
}

template <typename T>
__global__ void __launch_bounds__(kPencilThreads) k_zgreen_group(const __grid_constant__ ZGroup<T> g) {
  __shared__ double red[32][kNumRed];
  __shared__ int s_last;
  int m;
  const Cta cta = group_place(g.start, g.gx, g.n, &m);
  const ZArgs<T>& a = g.m[m];
  switch (a.HC <= pencil_max_hc(a.nz) ? a.nz : 0) {
    case 64: zgreen_cta<T, PencilSplit<64>::N1, PencilSplit<64>::N2>(a, cta, red, s_last); return;
    case 96: zgreen_cta<T, PencilSplit<96>::N1, PencilSplit<96>::N2>(a, cta, red, s_last); return;
    case 128: zgreen_cta<T, PencilSplit<128>::N1, PencilSplit<128>::N2>(a, cta, red, s_last); return;
    case 160: zgreen_cta<T, PencilSplit<160>::N1, PencilSplit<160>::N2>(a, cta, red, s_last); return;
    case 256: zgreen_cta<T, PencilSplit<256>::N1, PencilSplit<256>::N2>(a, cta, red, s_last); return;
    default: zgreen_cta<T, 0, 0>(a, cta, red, s_last); return;
  }
}

// Bound and exit of a group's device-side iteration loop: after `limit` executions of the
// loop body, or once every member's increment is decided, the loop condition is cleared.
// The execution count lives in the first member's status record.
struct GuardGroup {
  IterStatus* st[kMaxGroup];
  int n;
  int limit;
};
template <typename T>
__global__ void k_group_guard(const GuardGroup g, cudaGraphConditionalHandle cond) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int c = ++g.st[0]->guard;
    bool all = true;
    for (int m = 0; m < g.n; ++m) all = all && g.st[m]->done != 0;
    if (c >= g.limit || all) cudaGraphSetConditional(cond, 0u);
  }
}

// ---------------------------------------------------------------- small kernels -----
template <typename T, int NP>
__global__ void k_material_point(const MatDev<T> M, long long nvox, const T* __restrict__ R,
                                 const T* __restrict__ eps_n, const T* __restrict__ eps, T* state,
                                 T* sigma, T dt, int nsub, const T* __restrict__ root_tab) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw);  // kRootTabs
  if (NP != 0)
    for (int k = threadIdx.x; k < kRootTabs; k += blockDim.x) tab[k] = root_tab[k];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvox) return;
  const size_t n = (size_t)nvox;
  T r[9], en[6], e[6], s[6];
#pragma unroll
  for (int k = 0; k < 9; ++k) r[k] = R[(size_t)i * 9 + k];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    en[c] = eps_n[c * n + i];
    e[c] = eps[c * n + i];
  }
  MPState<T> y;
#pragma unroll
  for (int c = 0; c < 6; ++c) y.ep[c] = state[c * n + i];
#pragma unroll
  for (int c = 0; c < 16; ++c) y.v[c] = state[(6 + c) * n + i];
#pragma unroll
  for (int c = 0; c < 12; ++c) y.al[c] = state[(22 + c) * n + i];
  mc_voxel<T, NP>(M, r, en, e, y, dt, nsub, s, tab);
#pragma unroll
  for (int c = 0; c < 6; ++c) state[c * n + i] = y.ep[c];
#pragma unroll
  for (int c = 0; c < 16; ++c) state[(6 + c) * n + i] = y.v[c];
#pragma unroll
  for (int c = 0; c < 12; ++c) state[(22 + c) * n + i] = y.al[c];
#pragma unroll
  for (int c = 0; c < 6; ++c) sigma[c * n + i] = s[c];
}

// Stand-alone x transforms of ncomp real lines (FFT entry points): L lines of one
// component per CTA, packed in pairs (lines 2q, 2q + 1) as one complex sequence
// Z = A + iB at stride nx + 1 in shared memory, as in the x pass (register two-step
// transforms for the lengths of the PencilSplit table, Stockham passes otherwise); the
// forward transform keeps kx in [0, nx/2].
template <typename T>
struct XFftArgs {
  int nx, H, L, ncomp;
  long long NL;
  FftDim dx;
  const C2<T>* tw;
  const T* real;
  C2<T>* spec;
  T* real_out;
};

template <typename T, int SIGN>
__global__ void __launch_bounds__(kXThreads) k_xfft(const XFftArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = a.nx, xs = nx + 1;
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* b0 = tw + nx;
  C2<T>* b1 = b0 + (size_t)((a.L + 1) / 2) * xs;
  const int tid = threadIdx.x, nthr = blockDim.x, H = a.H, half = nx / 2;
  const long long line0 = (long long)blockIdx.x * a.L;
  const int nl = (int)min((long long)a.L, a.NL - line0);
  const int nq = (nl + 1) / 2;  // packed sequences (the last one holds one line when nl is odd)
  const int c = blockIdx.y;     // component
  const size_t nvox = (size_t)a.NL * nx;
  for (int i = tid; i < nx; i += nthr) tw[i] = a.tw[i];
  if (SIGN < 0) {
    const T* src = a.real + c * nvox + (size_t)line0 * nx;
    for (int t = tid; t < nq * nx; t += nthr) {
      const int q = t / nx, x = t - q * nx;
      const T re = src[(size_t)(2 * q) * nx + x];
      const T im = 2 * q + 1 < nl ? src[(size_t)(2 * q + 1) * nx + x] : T(0);
      b0[(size_t)q * xs + x] = mk<T>(re, im);
    }
    __syncthreads();
    C2<T>* r = xlines_fft<T, -1>(b0, b1, a.dx, nq, xs, tw, tid, nthr);
    // unpack: A = (Z_k + conj Z_{n-k}) / 2, B = (Z_k - conj Z_{n-k}) / (2i)
    for (int w = tid; w < nl * H; w += nthr) {
      const int l = w / H, xi = w - l * H;
      const int q = l >> 1;
      const C2<T> Z = r[(size_t)q * xs + xi];
      const C2<T> Zm = r[(size_t)q * xs + (xi == 0 ? 0 : nx - xi)];
      const C2<T> X = (l & 1) ? mk<T>(T(0.5) * (Z.y + Zm.y), T(-0.5) * (Z.x - Zm.x))
                              : mk<T>(T(0.5) * (Z.x + Zm.x), T(0.5) * (Z.y - Zm.y));
      a.spec[((size_t)c * a.NL + line0 + l) * H + xi] = X;
    }
  } else {
    // pack: Z_k = A_k + i B_k on the Hermitian-extended sequence (imaginary parts of the
    // kx = 0 and Nyquist entries dropped)
    for (int w = tid; w < nq * H; w += nthr) {
      const int q = w / H, xi = w - q * H;
      const size_t e0 = ((size_t)c * a.NL + line0 + 2 * q) * H + xi;
      C2<T> A = a.spec[e0];
      C2<T> B = 2 * q + 1 < nl ? a.spec[e0 + H] : mk<T>(T(0), T(0));
      if (xi == 0 || xi == half) {
        A.y = T(0);
        B.y = T(0);
      }
      C2<T>* seq = b0 + (size_t)q * xs;
      seq[xi] = mk<T>(A.x - B.y, A.y + B.x);
      if (xi > 0 && xi < half) seq[nx - xi] = mk<T>(A.x + B.y, B.x - A.y);
    }
    __syncthreads();
    C2<T>* r = xlines_fft<T, +1>(b0, b1, a.dx, nq, xs, tw, tid, nthr);
    T* dst = a.real_out + c * nvox + (size_t)line0 * nx;
    for (int t = tid; t < nl * nx; t += nthr) {
      const int l = t / nx, x = t - l * nx;
      const C2<T> z = r[(size_t)(l >> 1) * xs + x];
      dst[t] = (l & 1) ? z.y : z.x;
    }
  }
}

}  // namespace rve
