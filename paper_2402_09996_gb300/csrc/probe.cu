// ALU throughput probes: the measured denominators of the constitutive update's roofline.
//
// The per-voxel Meric-Cailletaud update (Sec. 3, with the regularised rates of Sec. 4) is
// bound by the plain FP32 (or FP64) FMA pipe and, for its logarithms and exponentials, by
// the MUFU unit -- not by tensor cores or HBM.  Each probe runs, per thread, kChains
// independent dependency chains of one operation, long enough that a launch lasts tens of
// milliseconds; the host times it with CUDA events and divides the operation count.
#include <cuda_runtime.h>

#include <string>

#include "../../include/rve.h"

namespace rve {
void set_global_error(const std::string& msg);
}

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;  // operations per chain per loop trip

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_probe_fma(int iters, T b, T c, T* sink) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == T(-1.25e-7)) sink[0] = s;  // keeps the chains alive; the values stay positive
}

// MUFU base-2 exponential: x -> 2^(-x) keeps every value in (1/2, 1].
__global__ void __launch_bounds__(kProbeThreads) k_probe_ex2(int iters, float* sink) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = float(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(a[k]) : "f"(-a[k]));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.25e-7f) sink[0] = s;
}

}  // namespace

extern "C" rve_status rve_alu_probe(int kind, int blocks, int iters, void* sink, void* stream, double* ops_out) {
  if (kind < 0 || kind > 2 || blocks < 1 || iters < 1 || !sink) {
    rve::set_global_error("rve_alu_probe: bad kind, size or NULL sink");
    return RVE_ERR_INVALID_ARG;
  }
  cudaStream_t s = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  const double lanes = (double)blocks * kProbeThreads;
  const double per_lane = (double)iters * kUnroll * kChains;
  if (kind == 0) {
    k_probe_fma<float><<<blocks, kProbeThreads, 0, s>>>(iters, 0.9999999f, 1e-7f, (float*)sink);
  } else if (kind == 1) {
    k_probe_fma<double><<<blocks, kProbeThreads, 0, s>>>(iters, 0.9999999, 1e-7, (double*)sink);
  } else {
    k_probe_ex2<<<blocks, kProbeThreads, 0, s>>>(iters, (float*)sink);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rve::set_global_error(std::string("rve_alu_probe: ") + cudaGetErrorString(e));
    return RVE_ERR_CUDA;
  }
  if (ops_out) *ops_out = lanes * per_lane * (kind == 2 ? 1.0 : 2.0);
  return RVE_OK;
}
