// Periodic Voronoi labelling with the centroid-plane twin split (input generation).
//
// Sec. 2.1: grain n is the set of points not farther from generator s_n than from any
// other generator, here on the periodic unit cell.  Labels are decided exactly:
// voxel centre ((i+1/2)/nx, ...), per-axis difference folded to [-1/2, 1/2]
// (d > 1/2 -> d - 1, then d < -1/2 -> d + 1), squared distance (dx*dx + dy*dy) + dz*dz
// with every operation rounded separately (no fused multiply-add), strict "<" while
// scanning generators in index order so ties go to the lowest index.
//
// Synthetic twins: a twinned parent p is cut by the plane through its centroid with
// normal n_p.  The centroid is (centre of the voxel holding s_p) + (integer sum of
// minimum-image voxel offsets) / count; a voxel goes to the twin (id n_parent + p)
// when (dx*n0 + dy*n1) + dz*n2 > 0 for its minimum-image offset from the centroid in
// voxel units (dx >= n/2 -> dx - n, dx < -n/2 -> dx + n).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rve.h"

namespace {

__device__ __forceinline__ double fold_unit(double d) {
  if (d > 0.5) d = __dadd_rn(d, -1.0);
  if (d < -0.5) d = __dadd_rn(d, 1.0);
  return d;
}

__global__ void k_voronoi(int nx, int ny, int nz, int n_seed, const double* __restrict__ seeds,
                          uint32_t* __restrict__ label) {
  const long long nvox = (long long)nx * ny * nz;
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox) return;
  const int i = (int)(v % nx);
  const int j = (int)((v / nx) % ny);
  const int k = (int)(v / ((long long)nx * ny));
  const double cx = __ddiv_rn(__dadd_rn((double)i, 0.5), (double)nx);
  const double cy = __ddiv_rn(__dadd_rn((double)j, 0.5), (double)ny);
  const double cz = __ddiv_rn(__dadd_rn((double)k, 0.5), (double)nz);
  double best = INFINITY;
  uint32_t lab = 0;
  for (int s = 0; s < n_seed; ++s) {
    const double dx = fold_unit(__dadd_rn(cx, -seeds[3 * s + 0]));
    const double dy = fold_unit(__dadd_rn(cy, -seeds[3 * s + 1]));
    const double dz = fold_unit(__dadd_rn(cz, -seeds[3 * s + 2]));
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (d2 < best) {
      best = d2;
      lab = (uint32_t)s;
    }
  }
  label[v] = lab;
}

__device__ __forceinline__ int wrap_int(int d, int n) {
  // minimum image in [-n/2, n/2)
  int r = (d + n / 2) % n;
  if (r < 0) r += n;
  return r - n / 2;
}

// Integer offset sums and counts of the twinned parents.
__global__ void k_centroid_sums(int nx, int ny, int nz, const uint32_t* __restrict__ label,
                                const uint8_t* __restrict__ twinned, const int* __restrict__ seed_vox,
                                unsigned long long* __restrict__ sums) {
  const long long nvox = (long long)nx * ny * nz;
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox) return;
  const uint32_t p = label[v];
  if (!twinned[p]) return;
  const int i = (int)(v % nx);
  const int j = (int)((v / nx) % ny);
  const int k = (int)(v / ((long long)nx * ny));
  const long long ox = wrap_int(i - seed_vox[3 * p + 0], nx);
  const long long oy = wrap_int(j - seed_vox[3 * p + 1], ny);
  const long long oz = wrap_int(k - seed_vox[3 * p + 2], nz);
  atomicAdd(&sums[4 * p + 0], (unsigned long long)ox);
  atomicAdd(&sums[4 * p + 1], (unsigned long long)oy);
  atomicAdd(&sums[4 * p + 2], (unsigned long long)oz);
  atomicAdd(&sums[4 * p + 3], 1ull);
}

__device__ __forceinline__ double fold_grid(double d, int n) {
  const double h = 0.5 * (double)n;
  if (d >= h) return __dadd_rn(d, -(double)n);
  if (d < -h) return __dadd_rn(d, (double)n);
  return d;
}

__global__ void k_twin_split(int nx, int ny, int nz, int n_parent, uint32_t* __restrict__ label,
                             const uint8_t* __restrict__ twinned, const double* __restrict__ cent,
                             const double* __restrict__ normal) {
  const long long nvox = (long long)nx * ny * nz;
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox) return;
  const uint32_t p = label[v];
  if (!twinned[p]) return;
  const int i = (int)(v % nx);
  const int j = (int)((v / nx) % ny);
  const int k = (int)(v / ((long long)nx * ny));
  const double dx = fold_grid(__dadd_rn(__dadd_rn((double)i, 0.5), -cent[3 * p + 0]), nx);
  const double dy = fold_grid(__dadd_rn(__dadd_rn((double)j, 0.5), -cent[3 * p + 1]), ny);
  const double dz = fold_grid(__dadd_rn(__dadd_rn((double)k, 0.5), -cent[3 * p + 2]), nz);
  const double side = __dadd_rn(__dadd_rn(__dmul_rn(dx, normal[3 * p + 0]), __dmul_rn(dy, normal[3 * p + 1])),
                                __dmul_rn(dz, normal[3 * p + 2]));
  if (side > 0.0) label[v] = (uint32_t)(n_parent + (int)p);
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

namespace rve {
void set_global_error(const std::string& msg);
}

#define LBL_CUDA(call)                                                      \
  do {                                                                      \
    cudaError_t _e = (call);                                                \
    if (_e != cudaSuccess) {                                                \
      rve::set_global_error(std::string("rve_label_voronoi: ") + #call + ": " + cudaGetErrorString(_e));     \
      return RVE_ERR_CUDA;                                                  \
    }                                                                       \
  } while (0)

extern "C" rve_status rve_label_voronoi(int nx, int ny, int nz, int n_parent, const double* seeds,
                                        const uint8_t* twinned, const double* twin_normal, uint32_t* out,
                                        int out_on_device, void* stream) {
  if (nx < 1 || ny < 1 || nz < 1 || n_parent < 1 || !seeds || !out) {
    rve::set_global_error("rve_label_voronoi: bad sizes or NULL pointer");
    return RVE_ERR_INVALID_ARG;
  }
  for (long long s = 0; s < 3LL * n_parent; ++s)
    if (!(seeds[s] >= 0.0 && seeds[s] < 1.0)) {
      rve::set_global_error("rve_label_voronoi: seeds must lie in [0, 1)");
      return RVE_ERR_INVALID_ARG;
    }
  const long long nvox = (long long)nx * ny * nz;
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  DevBuf d_seeds, d_label, d_tw, d_sv, d_sums, d_cent, d_nrm;
  LBL_CUDA(cudaMalloc(&d_seeds.p, 3 * sizeof(double) * n_parent));
  LBL_CUDA(cudaMemcpyAsync(d_seeds.p, seeds, 3 * sizeof(double) * n_parent, cudaMemcpyHostToDevice, st));
  uint32_t* lab = out;
  if (!out_on_device) {
    LBL_CUDA(cudaMalloc(&d_label.p, sizeof(uint32_t) * nvox));
    lab = (uint32_t*)d_label.p;
  }
  const int thr = 256;
  const unsigned grid = (unsigned)((nvox + thr - 1) / thr);
  k_voronoi<<<grid, thr, 0, st>>>(nx, ny, nz, n_parent, (const double*)d_seeds.p, lab);
  LBL_CUDA(cudaGetLastError());
  bool any_twin = false;
  if (twinned)
    for (int p = 0; p < n_parent; ++p) any_twin |= twinned[p] != 0;
  if (any_twin) {
    if (!twin_normal) {
      rve::set_global_error("rve_label_voronoi: twin_normal is NULL");
      return RVE_ERR_INVALID_ARG;
    }
    std::vector<int> sv(3 * n_parent);
    for (int p = 0; p < n_parent; ++p) {
      sv[3 * p + 0] = std::min((int)(seeds[3 * p + 0] * nx), nx - 1);
      sv[3 * p + 1] = std::min((int)(seeds[3 * p + 1] * ny), ny - 1);
      sv[3 * p + 2] = std::min((int)(seeds[3 * p + 2] * nz), nz - 1);
    }
    LBL_CUDA(cudaMalloc(&d_tw.p, n_parent));
    LBL_CUDA(cudaMemcpyAsync(d_tw.p, twinned, n_parent, cudaMemcpyHostToDevice, st));
    LBL_CUDA(cudaMalloc(&d_sv.p, sizeof(int) * 3 * n_parent));
    LBL_CUDA(cudaMemcpyAsync(d_sv.p, sv.data(), sizeof(int) * 3 * n_parent, cudaMemcpyHostToDevice, st));
    LBL_CUDA(cudaMalloc(&d_sums.p, sizeof(unsigned long long) * 4 * n_parent));
    LBL_CUDA(cudaMemsetAsync(d_sums.p, 0, sizeof(unsigned long long) * 4 * n_parent, st));
    k_centroid_sums<<<grid, thr, 0, st>>>(nx, ny, nz, lab, (const uint8_t*)d_tw.p, (const int*)d_sv.p,
                                          (unsigned long long*)d_sums.p);
    LBL_CUDA(cudaGetLastError());
    std::vector<unsigned long long> sums(4 * n_parent);
    LBL_CUDA(cudaMemcpyAsync(sums.data(), d_sums.p, sizeof(unsigned long long) * 4 * n_parent,
                             cudaMemcpyDeviceToHost, st));
    LBL_CUDA(cudaStreamSynchronize(st));
    std::vector<double> cent(3 * n_parent);
    for (int p = 0; p < n_parent; ++p) {
      const long long cnt = (long long)sums[4 * p + 3];
      for (int a = 0; a < 3; ++a) {
        const double base = (double)sv[3 * p + a] + 0.5;
        cent[3 * p + a] = cnt > 0 ? base + (double)(long long)sums[4 * p + a] / (double)cnt : base;
      }
    }
    LBL_CUDA(cudaMalloc(&d_cent.p, sizeof(double) * 3 * n_parent));
    LBL_CUDA(cudaMemcpyAsync(d_cent.p, cent.data(), sizeof(double) * 3 * n_parent, cudaMemcpyHostToDevice, st));
    LBL_CUDA(cudaMalloc(&d_nrm.p, sizeof(double) * 3 * n_parent));
    LBL_CUDA(cudaMemcpyAsync(d_nrm.p, twin_normal, sizeof(double) * 3 * n_parent, cudaMemcpyHostToDevice, st));
    k_twin_split<<<grid, thr, 0, st>>>(nx, ny, nz, n_parent, lab, (const uint8_t*)d_tw.p,
                                       (const double*)d_cent.p, (const double*)d_nrm.p);
    LBL_CUDA(cudaGetLastError());
  }
  if (!out_on_device) LBL_CUDA(cudaMemcpyAsync(out, lab, sizeof(uint32_t) * nvox, cudaMemcpyDeviceToHost, st));
  LBL_CUDA(cudaStreamSynchronize(st));
  return RVE_OK;
}

// ---------------------------------------------------------------------------------
// Labelling without device allocation.
//
// For callers that may not allocate device memory (a caller-owned memory pool, loops
// that cannot afford the device-wide synchronisation of cudaMalloc/cudaFree, embedding
// where allocation is forbidden), the scratch of the labelling lives in one static
// device array of fixed size; only the caller's output buffer is written besides it.
namespace {

constexpr int kNoAllocMax = RVE_NOALLOC_MAX_PARENTS;

struct NoAllocScratch {
  double seeds[3 * kNoAllocMax];
  double cent[3 * kNoAllocMax];
  double normal[3 * kNoAllocMax];
  unsigned long long sums[4 * kNoAllocMax];
  int seed_vox[3 * kNoAllocMax];
  uint8_t twinned[kNoAllocMax];
};

// Held by every GPU that loads this library until the process exits.  In host code the
// name is only a stand-in: kernels receive the device address looked up below.
static __device__ __align__(256) NoAllocScratch g_noalloc;

// Device address of g_noalloc per device ordinal, looked up once per device.
std::mutex g_noalloc_mu;
NoAllocScratch* g_noalloc_ptr[64] = {nullptr};

// Seed voxel indices: min(trunc(s * n), n - 1) per axis, as the host path computes them.
__global__ void k_seed_vox(int n_parent, int nx, int ny, int nz, NoAllocScratch* sc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_parent) return;
  const int n[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    const int v = (int)__dmul_rn(sc->seeds[3 * p + a], (double)n[a]);
    sc->seed_vox[3 * p + a] = v < n[a] - 1 ? v : n[a] - 1;
  }
}

// Centroid of each twinned parent: (seed voxel centre) + (integer offset sum) / count,
// the same rounded operations as the host path.
__global__ void k_centroids(int n_parent, NoAllocScratch* sc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_parent) return;
  const long long cnt = (long long)sc->sums[4 * p + 3];
  for (int a = 0; a < 3; ++a) {
    const double base = __dadd_rn((double)sc->seed_vox[3 * p + a], 0.5);
    sc->cent[3 * p + a] =
        cnt > 0 ? __dadd_rn(base, __ddiv_rn((double)(long long)sc->sums[4 * p + a], (double)cnt)) : base;
  }
}

}  // namespace

extern "C" rve_status rve_label_voronoi_noalloc(int nx, int ny, int nz, int n_parent, const double* seeds,
                                                const uint8_t* twinned, const double* twin_normal,
                                                uint32_t* out, void* stream) {
  if (nx < 1 || ny < 1 || nz < 1 || n_parent < 1 || !seeds || !out) {
    rve::set_global_error("rve_label_voronoi_noalloc: bad sizes or NULL pointer");
    return RVE_ERR_INVALID_ARG;
  }
  if (n_parent > kNoAllocMax) {
    rve::set_global_error("rve_label_voronoi_noalloc: n_parent " + std::to_string(n_parent) +
                          " exceeds the no-allocation maximum of " + std::to_string(kNoAllocMax));
    return RVE_ERR_INVALID_ARG;
  }
  for (long long s = 0; s < 3LL * n_parent; ++s)
    if (!(seeds[s] >= 0.0 && seeds[s] < 1.0)) {
      rve::set_global_error("rve_label_voronoi_noalloc: seeds must lie in [0, 1)");
      return RVE_ERR_INVALID_ARG;
    }
  bool any_twin = false;
  if (twinned)
    for (int p = 0; p < n_parent; ++p) any_twin |= twinned[p] != 0;
  if (any_twin && !twin_normal) {
    rve::set_global_error("rve_label_voronoi_noalloc: twin_normal is NULL");
    return RVE_ERR_INVALID_ARG;
  }
  int dev = 0;
  LBL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    rve::set_global_error("rve_label_voronoi_noalloc: device ordinal out of range");
    return RVE_ERR_INVALID_ARG;
  }
  NoAllocScratch* sc = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      LBL_CUDA(cudaGetSymbolAddress(&p, g_noalloc));
      g_noalloc_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    sc = g_noalloc_ptr[dev];
  }
  const long long nvox = (long long)nx * ny * nz;
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  LBL_CUDA(cudaMemcpyAsync(sc->seeds, seeds, 3 * sizeof(double) * n_parent, cudaMemcpyHostToDevice, st));
  const int thr = 256;
  const unsigned grid = (unsigned)((nvox + thr - 1) / thr);
  k_voronoi<<<grid, thr, 0, st>>>(nx, ny, nz, n_parent, sc->seeds, out);
  LBL_CUDA(cudaGetLastError());
  if (any_twin) {
    const unsigned pg = (unsigned)((n_parent + 127) / 128);
    LBL_CUDA(cudaMemcpyAsync(sc->twinned, twinned, n_parent, cudaMemcpyHostToDevice, st));
    LBL_CUDA(cudaMemcpyAsync(sc->normal, twin_normal, 3 * sizeof(double) * n_parent, cudaMemcpyHostToDevice, st));
    // the array keeps the previous call's contents: the sums must start at zero
    LBL_CUDA(cudaMemsetAsync(sc->sums, 0, 4 * sizeof(unsigned long long) * n_parent, st));
    k_seed_vox<<<pg, 128, 0, st>>>(n_parent, nx, ny, nz, sc);
    LBL_CUDA(cudaGetLastError());
    k_centroid_sums<<<grid, thr, 0, st>>>(nx, ny, nz, out, sc->twinned, sc->seed_vox, sc->sums);
    LBL_CUDA(cudaGetLastError());
    k_centroids<<<pg, 128, 0, st>>>(n_parent, sc);
    LBL_CUDA(cudaGetLastError());
    k_twin_split<<<grid, thr, 0, st>>>(nx, ny, nz, n_parent, out, sc->twinned, sc->cent, sc->normal);
    LBL_CUDA(cudaGetLastError());
  }
  LBL_CUDA(cudaStreamSynchronize(st));
  return RVE_OK;
}
