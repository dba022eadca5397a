// C ABI and host-side driver of the Green-operator fixed-point solver.
//
// The increment loop (paper Sec. 5: quasi-static strain steps) runs on the host; each
// fixed-point iteration is four kernel launches on the handle's stream (see
// solver_kernels.cuh) followed by one read of a small status record.  All arithmetic on
// fields happens in the kernels; the host only forms the 6-component macroscopic
// increment and decides convergence from values the kernels computed in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/rve.h"
#include "launch.h"
#include "solver_kernels.cuh"

using namespace rve;

namespace {

thread_local std::string g_err;

constexpr double kPi = 3.14159265358979323846;
const double kMw[6] = {1.0, 1.0, 1.0, 1.41421356237309504880, 1.41421356237309504880, 1.41421356237309504880};

bool factor_radices(int n, FftDim* d) {
  if (n < 1 || n > 512) return false;
  d->n = n;
  d->nst = 0;
  int m = n;
  while (m % 4 == 0) { d->radix[d->nst++] = 4; m /= 4; }
  while (m % 2 == 0) { d->radix[d->nst++] = 2; m /= 2; }
  while (m % 3 == 0) { d->radix[d->nst++] = 3; m /= 3; }
  while (m % 5 == 0) { d->radix[d->nst++] = 5; m /= 5; }
  return m == 1 && d->nst <= 12;
}

// Jacobi eigenvalues of a symmetric 6x6 matrix (host, for the reference medium).
void sym_eigvals6(const double A_in[36], double ev[6]) {
  double A[36];
  std::memcpy(A, A_in, sizeof(A));
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < 6; ++p)
      for (int q = p + 1; q < 6; ++q) off += A[p * 6 + q] * A[p * 6 + q];
    if (off < 1e-30) break;
    for (int p = 0; p < 6; ++p)
      for (int q = p + 1; q < 6; ++q) {
        const double apq = A[p * 6 + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (A[q * 6 + q] - A[p * 6 + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 6; ++k) {
          const double akp = A[k * 6 + p], akq = A[k * 6 + q];
          A[k * 6 + p] = c * akp - s * akq;
          A[k * 6 + q] = s * akp + c * akq;
        }
        for (int k = 0; k < 6; ++k) {
          const double apk = A[p * 6 + k], aqk = A[q * 6 + k];
          A[p * 6 + k] = c * apk - s * aqk;
          A[q * 6 + k] = s * apk + c * aqk;
        }
      }
  }
  for (int i = 0; i < 6; ++i) ev[i] = A[i * 6 + i];
}

// In-place inverse of an n x n matrix (Gauss-Jordan with partial pivoting).
bool invert(double* M, int n) {
  std::vector<double> a(M, M + n * n), inv(n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[r * n + c]) > std::fabs(a[piv * n + c])) piv = r;
    if (std::fabs(a[piv * n + c]) < 1e-300) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[c * n + k], a[piv * n + k]);
        std::swap(inv[c * n + k], inv[piv * n + k]);
      }
    const double d = a[c * n + c];
    for (int k = 0; k < n; ++k) {
      a[c * n + k] /= d;
      inv[c * n + k] /= d;
    }
    for (int r = 0; r < n; ++r)
      if (r != c) {
        const double f = a[r * n + c];
        if (f == 0.0) continue;
        for (int k = 0; k < n; ++k) {
          a[r * n + k] -= f * a[c * n + k];
          inv[r * n + k] -= f * inv[c * n + k];
        }
      }
  }
  std::memcpy(M, inv.data(), sizeof(double) * n * n);
  return true;
}

void bunge(const double* e, double R[9]) {
  const double c1 = std::cos(e[0]), s1 = std::sin(e[0]);
  const double c = std::cos(e[1]), s = std::sin(e[1]);
  const double c2 = std::cos(e[2]), s2 = std::sin(e[2]);
  // Rz(phi1) Rx(Phi) Rz(phi2), crystal -> sample
  R[0] = c1 * c2 - s1 * c * s2;
  R[1] = -c1 * s2 - s1 * c * c2;
  R[2] = s1 * s;
  R[3] = s1 * c2 + c1 * c * s2;
  R[4] = -s1 * s2 + c1 * c * c2;
  R[5] = -c1 * s;
  R[6] = s * s2;
  R[7] = s * c2;
  R[8] = c;
}

// d R / d (phi1, Phi, phi2) of `bunge`, entry-wise (dR[k][i] = d R[i] / d e[k]).
void bunge_grad(const double* e, double dR[3][9]) {
  const double c1 = std::cos(e[0]), s1 = std::sin(e[0]);
  const double c = std::cos(e[1]), s = std::sin(e[1]);
  const double c2 = std::cos(e[2]), s2 = std::sin(e[2]);
  const double d1[9] = {-s1 * c2 - c1 * c * s2, s1 * s2 - c1 * c * c2, c1 * s, c1 * c2 - s1 * c * s2,
                        -c1 * s2 - s1 * c * c2, s1 * s, 0.0, 0.0, 0.0};
  const double d2[9] = {s1 * s * s2, s1 * s * c2, s1 * c, -c1 * s * s2, -c1 * s * c2, -c1 * c, c * s2, c * c2, -s};
  const double d3[9] = {-c1 * s2 - s1 * c * c2, -c1 * c2 + s1 * c * s2, 0.0, -s1 * s2 + c1 * c * c2,
                        -s1 * c2 - c1 * c * s2, 0.0, s * c2, -s * s2, 0.0};
  for (int i = 0; i < 9; ++i) {
    dR[0][i] = d1[i];
    dR[1][i] = d2[i];
    dR[2][i] = d3[i];
  }
}

// Isotropic reference medium: 3 k0 = 2 mu0 = (min + max Mandel eigenvalue of C) / 2.
void reference_medium(const rve_material& m, double* lam0, double* mu0) {
  double A[36] = {0};
  A[0] = A[7] = m.C11;
  A[14] = m.C33;
  A[1] = A[6] = m.C12;
  A[2] = A[12] = A[8] = A[13] = m.C13;
  A[21] = 2.0 * m.C44;
  A[28] = 2.0 * m.C44;
  A[35] = 2.0 * m.C66;
  double ev[6];
  sym_eigvals6(A, ev);
  const double lo = *std::min_element(ev, ev + 6), hi = *std::max_element(ev, ev + 6);
  const double two_mu = 0.5 * (lo + hi);
  *mu0 = 0.5 * two_mu;
  *lam0 = two_mu / 3.0 - 2.0 * (*mu0) / 3.0;
}

// The handle's reference medium: the caller's (opt.c0_lambda, opt.c0_mu) when c0_mu > 0,
// else reference_medium's rule.
void set_reference_medium(const rve_options& o, const rve_material& m, double* lam0, double* mu0) {
  if (o.c0_mu > 0.0) {
    *lam0 = o.c0_lambda;
    *mu0 = o.c0_mu;
  } else {
    reference_medium(m, lam0, mu0);
  }
}

void c0_mandel(double lam, double mu, double M[36]) {
  std::memset(M, 0, 36 * sizeof(double));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i * 6 + j] = lam + (i == j ? 2.0 * mu : 0.0);
  for (int i = 3; i < 6; ++i) M[i * 6 + i] = 2.0 * mu;
}

int is_small_int(double x) {
  const double r = std::round(x);
  return (std::fabs(x - r) == 0.0 && r >= 1.0 && r <= 64.0) ? (int)r : 0;
}

// m = 1 / log2(1/u1) with u1^n + u1 = 1 (bisection): the exponent that makes the
// smooth minimum (1 + beta^m)^(-1/m) exact at beta = 1 for the rate root's start.
double smooth_min_exponent(double n) {
  double lo = 0.0, hi = 1.0;
  for (int i = 0; i < 200; ++i) {
    const double mid = 0.5 * (lo + hi);
    if (std::pow(mid, n) + mid - 1.0 > 0.0) hi = mid;
    else lo = mid;
  }
  return 1.0 / std::log2(1.0 / (0.5 * (lo + hi)));
}

// Iterations enqueued per host synchronisation (launches after convergence return at
// once), and event slots for per-launch timing: 4 kernels per iteration + shift + commit.
constexpr int kBatch = 8;
constexpr int kTSlots = 4 * kBatch + 2;
constexpr int kSlotShift = 4 * kBatch;
constexpr int kSlotCommit = 4 * kBatch + 1;

int default_nsub(double dt) {
  int n = 1;
  while (dt / n > 0.125 * (1.0 + 1e-12) && n < (1 << 20)) n *= 2;
  return n;
}

}  // namespace

struct rve_s {
  int nx = 0, ny = 0, nz = 0, H = 0;
  long long nvox = 0, NL = 0;
  int n_grains = 0;
  rve_options opt{};
  rve_material mat{};
  double Edot[6] = {0, 0, 1e-3, 0, 0, 0};
  uint8_t ctrl[6] = {0, 0, 1, 0, 0, 0};
  double Sigma[6] = {0, 0, 0, 0, 0, 0};
  double dt = 1.0;
  cudaStream_t stream = nullptr;
  int tsize = 8;
  FftDim dx{}, dy{}, dz{};
  std::vector<double> euler;
  // device buffers
  // Three strain spectra and three tau_hat spectra rotate during an increment; the
  // committed pair (spec[sb]: strain at t_n, P[pb]: the tau_hat that produced it) is
  // never written before the commit, so a failed increment leaves them intact.
  void* spec[3] = {nullptr, nullptr, nullptr};
  void* P[3] = {nullptr, nullptr, nullptr};
  int sb = 0, pb = 0;
  void* backup = nullptr;
  double* dhist = nullptr;  // device (e_eq, c_F) history, 2 * max_iter
  void *ep = nullptr, *v = nullptr, *al = nullptr, *eps_n = nullptr, *sig_n = nullptr;
  unsigned char* flow = nullptr;  // x pass: per warp of 32 voxels, flowed in iteration 0 (XArgs::flow)
  uint32_t* grain = nullptr;
  void* Rg = nullptr;
  void* root_tab = nullptr;  // kRootTabs rate-root table values (slip systems, twin exponent)
  void *tw_x = nullptr, *tw_y = nullptr, *tw_z = nullptr;
  void *kx = nullptr, *ky = nullptr, *kz = nullptr;
  double* partial = nullptr;
  unsigned int* counter = nullptr;
  IterStatus* st = nullptr;
  IterStatus* st_host = nullptr;  // pinned
  std::vector<void*> owned;
  // launch geometry
  int L = 1, xgrid = 0;
  size_t xsmem = 0, ysmem = 0, zsmem = 0;
  int yHC = 1, zHC = 1;
  int xs = 0;  // x-pass shared-memory line stride
  double lam0 = 0, mu0 = 0;
  // host state
  double E_n[6] = {0}, E_prev[6] = {0};
  double time = 0.0;
  int increment = 0;
  std::vector<rve_effective> hist;
  std::string err;
  // optional per-kernel event timing
  cudaEvent_t ev_a[kTSlots] = {}, ev_b[kTSlots] = {};
  int ev_kind[kTSlots] = {};
  bool ev_used[kTSlots] = {};
  double k_ms[RVE_K_COUNT] = {};
  long long k_n[RVE_K_COUNT] = {};
  std::vector<double> res_e, res_c;  // convergence history of the latest increment
  // resumable increment (shared by rve_step and rve_step_batch): the host enqueues a
  // phase of work, records ev_sync after the status copy, and resumes when it completes
  cudaEvent_t ev_sync = nullptr;
  int inc_phase = 0;  // 0 idle, 1 fixed-point iterations in flight, 2 commit in flight
  int inc_it0 = 0, inc_nb = 0, inc_last = 0;
  double inc_dE0[6] = {0, 0, 0, 0, 0, 0};
  double inc_E[6] = {0, 0, 0, 0, 0, 0};
  double inc_e = 0.0, inc_c = 0.0;
  // device-side increment loops (opt.graphs): one executable graph per buffer rotation
  cudaGraph_t graph[3] = {nullptr, nullptr, nullptr};
  cudaGraphExec_t gexec[3] = {nullptr, nullptr, nullptr};
  cudaStream_t cap[2] = {nullptr, nullptr};  // capture streams
  // adjoint of an increment (rve_adjoint_increment): host grain map, scratch, and the
  // x pass's linear-law mode (s = B eps - g) used by the adjoint fixed point
  std::vector<uint32_t> gid_host;
  void* adj = nullptr;  // one block of per-voxel scratch arrays, type by precision
  void* adj_perm = nullptr;  // voxel indices sorted by grain (increasing within a grain)
  void* adj_goff = nullptr;  // n_grains + 1 offsets into adj_perm
  bool lin_mode = false;
  const void* lin_B = nullptr;
  const void* lin_g = nullptr;
  void* lin_mu = nullptr;
  double lin_sref = 0.0;  // source scale of the adjoint fixed point (floor of the error norms)
  // FFT tile autotuner (opt.autotune): runs once, before the first increment
  bool tuned = false;
  IterStatus* st_tune = nullptr;  // scratch status and history for timing the z pass
  double* hist_tune = nullptr;
};

namespace {

// A named NVTX range over a scope (an increment, a batch, an adjoint increment): profilers
// attach the kernels launched inside it to the name (ncu --nvtx, nsys); without an
// attached tool a push or pop does nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

rve_status fail(rve_s* h, rve_status s, const std::string& msg) {
  if (h) h->err = msg;
  g_err = msg;
  return s;
}

rve_status cuda_fail(rve_s* h, cudaError_t e, const char* where) {
  return fail(h, RVE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define RVE_CUDA(h, call)                                   \
  do {                                                      \
    cudaError_t _e = (call);                                \
    if (_e != cudaSuccess) return cuda_fail((h), _e, #call); \
  } while (0)

rve_status dalloc(rve_s* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (h->opt.alloc) {
    *p = h->opt.alloc(bytes, h->opt.alloc_ctx);
    if (!*p) return fail(h, RVE_ERR_OOM, "allocator callback returned NULL");
  } else {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(h, RVE_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  h->owned.push_back(*p);
  return RVE_OK;
}

// Per-launch event timing (opt.timing): a launch records into an event slot; after the
// next stream synchronisation tcollect folds the slots into per-kind totals.
void tstart(rve_s* h, int slot, int kind) {
  if (!h->opt.timing) return;
  cudaEventRecord(h->ev_a[slot], h->stream);
  h->ev_kind[slot] = kind;
}
void tstop(rve_s* h, int slot) {
  if (!h->opt.timing) return;
  cudaEventRecord(h->ev_b[slot], h->stream);
  h->ev_used[slot] = true;
}
// work_iters: iterations of the batch that did work; launches of later iterations returned
// at once and are counted as RVE_K_IDLE.
void tcollect(rve_s* h, int work_iters) {
  if (!h->opt.timing) return;
  for (int k = 0; k < kTSlots; ++k)
    if (h->ev_used[k]) {
      if (k < kSlotShift && k / 4 >= work_iters) {
        h->k_n[RVE_K_IDLE] += 1;
      } else {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev_a[k], h->ev_b[k]) == cudaSuccess) {
          h->k_ms[h->ev_kind[k]] += ms;
          h->k_n[h->ev_kind[k]] += 1;
        }
      }
      h->ev_used[k] = false;
    }
}

void drop_graphs(rve_s* h) {
  for (int k = 0; k < 3; ++k) {
    if (h->gexec[k]) cudaGraphExecDestroy(h->gexec[k]);
    if (h->graph[k]) cudaGraphDestroy(h->graph[k]);
    h->gexec[k] = nullptr;
    h->graph[k] = nullptr;
  }
}

void release(rve_s* h) {
  drop_graphs(h);
  for (int k = 0; k < 2; ++k) {
    if (h->cap[k]) cudaStreamDestroy(h->cap[k]);
    h->cap[k] = nullptr;
  }
  if (h->ev_sync) cudaEventDestroy(h->ev_sync);
  h->ev_sync = nullptr;
  for (int k = 0; k < kTSlots; ++k) {
    if (h->ev_a[k]) cudaEventDestroy(h->ev_a[k]);
    if (h->ev_b[k]) cudaEventDestroy(h->ev_b[k]);
    h->ev_a[k] = h->ev_b[k] = nullptr;
  }
  for (void* p : h->owned) {
    if (h->opt.free) h->opt.free(p, h->opt.alloc_ctx);
    else cudaFree(p);
  }
  h->owned.clear();
  if (h->st_host) cudaFreeHost(h->st_host);
  h->st_host = nullptr;
}

// The x pass stages the two rate-root tables (kRootTabs values) in shared memory after
// its FFT buffers.
size_t xsmem_total(const rve_s* h) {
  const size_t elem = h->opt.precision == RVE_FP64 ? sizeof(double) : sizeof(float);
  return h->xsmem + (size_t)kRootTabs * elem;
}

template <typename T>
MatDev<T> make_mat(const rve_s* h) {
  const rve_material& m = h->mat;
  MatDev<T> M;
  M.C11 = (T)m.C11; M.C12 = (T)m.C12; M.C13 = (T)m.C13; M.C33 = (T)m.C33; M.C44 = (T)m.C44; M.C66 = (T)m.C66;
  const char kinds[12] = {'s', 's', 'o', 's', 's', 'o', 's', 's', 'o', 's', 's', 'o'};
  for (int s = 0; s < 12; ++s) M.r0[s] = (T)(kinds[s] == 'o' ? m.r0_ord : m.r0_sup);
  for (int s = 12; s < 16; ++s) M.r0[s] = (T)m.r0_twin;
  M.K = (T)m.K; M.n = (T)m.n; M.Kt = (T)m.Kt; M.nt = (T)m.nt;
  M.Q_s = (T)m.Q_s; M.Q_b = (T)m.Q_b; M.b_s = (T)m.b_s; M.b_b = (T)m.b_b;
  M.h_diag = (T)m.h_diag; M.h_off = (T)m.h_off; M.c = (T)m.c; M.d = (T)m.d;
  M.Kc = (T)m.Kc; M.fm = (T)m.fm; M.eta = (T)m.eta;
  M.n_int = is_small_int(m.n);
  M.nt_int = is_small_int(m.nt);
  M.lam0 = (T)h->lam0;
  M.mu0 = (T)h->mu0;
  M.inv_n = (T)(1.0 / m.n);
  M.inv_nt = (T)(1.0 / m.nt);
  M.sm = (T)smooth_min_exponent(m.n);
  M.smt = (T)smooth_min_exponent(m.nt);
  M.lg_K = (T)std::log2(m.K);
  M.lg_Kt = (T)std::log2(m.Kt);
  M.lg_eta = (T)(m.eta > 0 ? std::log2(m.eta) : 0.0);
  const double sc = 1.0 / std::sqrt(6.0);
  M.C11s = (T)(m.C11 * sc); M.C12s = (T)(m.C12 * sc); M.C13s = (T)(m.C13 * sc); M.C33s = (T)(m.C33 * sc);
  M.C44s2 = (T)(2.0 * m.C44 * sc); M.C66s2 = (T)(2.0 * m.C66 * sc);
  return M;
}

rve_status check_material(rve_s* h, const rve_material& m) {
  const double vals[] = {m.C11, m.C12, m.C13, m.C33, m.C44, m.C66, m.r0_ord, m.r0_sup, m.r0_twin, m.K, m.n, m.Kt,
                         m.nt, m.Q_s, m.Q_b, m.b_s, m.b_b, m.h_diag, m.h_off, m.c, m.d, m.Kc, m.fm, m.eta};
  for (double x : vals)
    if (!std::isfinite(x)) return fail(h, RVE_ERR_INVALID_ARG, "material constant is not finite");
  if (m.K <= 0 || m.Kt <= 0 || m.n < 1 || m.nt < 1 || m.eta < 0)
    return fail(h, RVE_ERR_INVALID_ARG, "need K, Kt > 0, n, nt >= 1 and eta >= 0");
  // positive definite stiffness: the Mandel eigenvalues must be positive
  double A[36] = {0};
  A[0] = A[7] = m.C11;
  A[14] = m.C33;
  A[1] = A[6] = m.C12;
  A[2] = A[12] = A[8] = A[13] = m.C13;
  A[21] = A[28] = 2.0 * m.C44;
  A[35] = 2.0 * m.C66;
  double ev[6];
  sym_eigvals6(A, ev);
  for (double e : ev)
    if (!(e > 0)) return fail(h, RVE_ERR_INVALID_ARG, "elastic stiffness is not positive definite");
  return RVE_OK;
}

// Twiddles e^{-2 pi i m / n}, m = 0 .. n - 1, as interleaved (re, im) pairs at out.
template <typename T>
void fill_twiddles(int n, T* out) {
  for (int m = 0; m < n; ++m) {
    const double a = 2.0 * kPi * (double)m / (double)n;
    out[2 * m] = (T)std::cos(a);
    out[2 * m + 1] = (T)(-std::sin(a));
  }
}

template <typename T>
rve_status upload_tables(rve_s* h) {
  auto tw = [&](int n, void** dst) -> rve_status {
    std::vector<T> t(2 * n);
    fill_twiddles<T>(n, t.data());
    rve_status s = dalloc(h, dst, t.size() * sizeof(T));
    if (s) return s;
    RVE_CUDA(h, cudaMemcpyAsync(*dst, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    RVE_CUDA(h, cudaStreamSynchronize(h->stream));
    return RVE_OK;
  };
  rve_status s;
  if ((s = tw(h->nx, &h->tw_x))) return s;
  if ((s = tw(h->ny, &h->tw_y))) return s;
  if ((s = tw(h->nz, &h->tw_z))) return s;
  // wave-vector tables per dimension
  auto kt = [&](int n, int count, void** dst) -> rve_status {
    std::vector<T> t(2 * count);
    for (int i = 0; i < count; ++i) {
      if (h->opt.green == RVE_GREEN_WILLOT) {
        // sin and cos of pi i / n, exact at the Nyquist index (cos = 0, so kappa vanishes
        // where two or more components sit at Nyquist)
        const double a = kPi * (double)i / (double)n;
        t[2 * i] = (T)(2 * i == n ? 1.0 : std::sin(a));
        t[2 * i + 1] = (T)(2 * i == n ? 0.0 : std::cos(a));
      } else {
        double f = (i <= n / 2) ? (double)i : (double)(i - n);
        if (n % 2 == 0 && i == n / 2) f = 0.0;
        t[2 * i] = (T)(2.0 * kPi * f / (double)n);
        t[2 * i + 1] = (T)0;
      }
    }
    rve_status s2 = dalloc(h, dst, t.size() * sizeof(T));
    if (s2) return s2;
    RVE_CUDA(h, cudaMemcpyAsync(*dst, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    RVE_CUDA(h, cudaStreamSynchronize(h->stream));
    return RVE_OK;
  };
  if ((s = kt(h->nx, h->H, &h->kx))) return s;
  if ((s = kt(h->ny, h->ny, &h->ky))) return s;
  if ((s = kt(h->nz, h->nz, &h->kz))) return s;
  // per-grain rotations
  std::vector<T> Rg((size_t)h->n_grains * 9);
  for (int g = 0; g < h->n_grains; ++g) {
    double R[9];
    bunge(&h->euler[3 * g], R);
    for (int i = 0; i < 9; ++i) Rg[(size_t)g * 9 + i] = (T)R[i];
  }
  if ((s = dalloc(h, &h->Rg, Rg.size() * sizeof(T)))) return s;
  RVE_CUDA(h, cudaMemcpyAsync(h->Rg, Rg.data(), Rg.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

// Dynamic shared memory of the y pass (twiddles + two buffers of HC*6 padded lines) and of
// the z pass (the same + HC*nz residual terms).
template <typename T>
size_t y_smem(const rve_s* h, int hc) {
  return (size_t)(h->ny + 12 * hc * (h->ny + 1)) * 2 * sizeof(T);
}
template <typename T>
size_t z_smem(const rve_s* h, int hc) {
  return (size_t)(h->nz + 12 * hc * (h->nz + 1)) * 2 * sizeof(T) + (size_t)hc * h->nz * sizeof(double);
}

template <typename T>
rve_status alloc_fields(rve_s* h) {
  const size_t spec = (size_t)6 * h->NL * h->H * 2 * sizeof(T);
  const size_t fld = (size_t)h->nvox * sizeof(T);
  rve_status s;
  void** bufs[] = {&h->spec[0], &h->spec[1], &h->spec[2], &h->P[0], &h->P[1], &h->P[2]};
  for (void** b : bufs) {
    if ((s = dalloc(h, b, spec))) return s;
    RVE_CUDA(h, cudaMemsetAsync(*b, 0, spec, h->stream));
  }
  if ((s = dalloc(h, &h->backup, (size_t)6 * h->NL * 2 * sizeof(T)))) return s;
  struct {
    void** p;
    int comps;
  } fl[] = {{&h->ep, 6}, {&h->v, 16}, {&h->al, 12}, {&h->eps_n, 6}, {&h->sig_n, 6}};
  for (auto& f : fl) {
    if ((s = dalloc(h, f.p, fld * f.comps))) return s;
    RVE_CUDA(h, cudaMemsetAsync(*f.p, 0, fld * f.comps, h->stream));
  }
  {
    const size_t nflow = (size_t)(h->nvox + 31) / 32;
    if ((s = dalloc(h, (void**)&h->flow, nflow))) return s;
    RVE_CUDA(h, cudaMemsetAsync(h->flow, 0, nflow, h->stream));
  }
  // launch geometry
  // x lines per CTA: enough to give every thread a voxel, up to 4 voxels per thread (a
  // thread then integrates voxels of several lines, which evens out the elastic/plastic
  // work between the CTA's warps) while keeping at least 2 CTAs per SM
  {
    const long long fill = (x_threads() + h->nx - 1) / h->nx;
    const long long most = std::max<long long>(1, 4LL * x_threads() / h->nx);
    const long long keep = std::max<long long>(1, h->NL / (2 * 152));
    h->L = (int)std::max(fill, std::min(most, keep));
  }
  h->xgrid = (int)((h->NL + h->L - 1) / h->L);
  // x sequences in shared memory: odd stride nx + 1 for the register transforms of the
  // lengths with a two-step split (conflict-free steps), nx for the Stockham passes
  h->xs = pencil_n1(h->nx) > 0 ? h->nx + 1 : h->nx;
  h->xsmem = (size_t)(h->nx + 6 * h->L * h->xs) * 2 * sizeof(T);  // FFT buffers; + tables: xsmem_total
  // y and z passes: tiles of HC kx values x 6 components (two buffers of padded lines);
  // default about 50 KB per CTA so that four CTAs share an SM (the autotuner may change it)
  const size_t tile_budget = 50 * 1024;
  h->yHC = (int)std::max<size_t>(1, std::min<size_t>(16, tile_budget / (2 * 6 * 2 * sizeof(T) * (h->ny + 1))));
  h->zHC = (int)std::max<size_t>(1, std::min<size_t>(16, tile_budget / (2 * 6 * 2 * sizeof(T) * (h->nz + 1))));
  if (h->opt.y_tile > 0) h->yHC = h->opt.y_tile;
  if (h->opt.z_tile > 0) h->zHC = h->opt.z_tile;
  h->yHC = std::min(h->yHC, h->H);
  h->zHC = std::min(h->zHC, h->H);
  // lines with a two-step split run the register transforms at every width: clamp to their limit
  if (pencil_max_hc(h->ny) > 0) h->yHC = std::min(h->yHC, pencil_max_hc(h->ny));
  if (pencil_max_hc(h->nz) > 0) h->zHC = std::min(h->zHC, pencil_max_hc(h->nz));
  h->ysmem = y_smem<T>(h, h->yHC);
  h->zsmem = z_smem<T>(h, h->zHC);
  // x-pass partials per CTA; z-pass partials per (ky, kx) column
  const size_t npart = std::max((size_t)h->xgrid * kNumRed, (size_t)h->ny * h->H);
  if ((s = dalloc(h, (void**)&h->partial, npart * sizeof(double)))) return s;
  if ((s = dalloc(h, (void**)&h->counter, 64))) return s;
  RVE_CUDA(h, cudaMemsetAsync(h->counter, 0, 64, h->stream));
  if ((s = dalloc(h, (void**)&h->st, sizeof(IterStatus)))) return s;
  RVE_CUDA(h, cudaMemsetAsync(h->st, 0, sizeof(IterStatus), h->stream));
  RVE_CUDA(h, cudaMallocHost((void**)&h->st_host, sizeof(IterStatus)));
  const int max_iter = h->opt.max_iter > 0 ? h->opt.max_iter : 1000;
  if ((s = dalloc(h, (void**)&h->dhist, (size_t)2 * max_iter * sizeof(double)))) return s;
  if ((s = dalloc(h, (void**)&h->st_tune, sizeof(IterStatus)))) return s;
  RVE_CUDA(h, cudaMemsetAsync(h->st_tune, 0, sizeof(IterStatus), h->stream));
  if ((s = dalloc(h, (void**)&h->hist_tune, 2 * sizeof(double)))) return s;
  return RVE_OK;
}

// Root table of the regularised rate (constitutive.cuh, reg_rate_tab) for exponent n:
// D = log2 u*, u* in (0, 1] the root of u^n + 2^x u = 1 (bisection to double precision),
// on the nodes x_k = -kRootSpan + k / kRootPerUnit, k = 0..kRootIv, stored per interval
// as the line through its two end nodes, D = a_i + b_i t with t = (x + kRootSpan)
// kRootPerUnit - 1/2.  The kink of the asymptotes min(0, -x) sits on the node x = 0, so
// every interval is smooth.
void root_table(double n, double* out) {
  std::vector<double> D(kRootIv + 1);
  for (int k = 0; k <= kRootIv; ++k) {
    const double x = -kRootSpan + (double)k / kRootPerUnit;
    const double beta = std::exp2(x);
    double lo = 0.0, hi = 1.0;
    for (int i = 0; i < 200; ++i) {
      const double mid = 0.5 * (lo + hi);
      if (std::pow(mid, n) + beta * mid - 1.0 > 0.0) hi = mid;
      else lo = mid;
    }
    D[k] = std::log2(0.5 * (lo + hi));
  }
  for (int i = 0; i < kRootIv; ++i) {
    const double b = D[i + 1] - D[i];
    out[2 * i] = D[i] + b * (0.5 - (double)i);
    out[2 * i + 1] = b;
  }
}

// The two tables of a material: the slip systems' lines in log2 a (P = 1, so the
// coefficients of constitutive.cuh root_coef are constants: alpha_i = b1 + a_i + b_i b2,
// beta_i = a1 + b_i a2), then the twin exponent's lines in the table coordinate t.
template <typename T>
std::vector<T> root_tables(const rve_material& m) {
  std::vector<double> d(kRootTabs, 0.0);
  root_table(m.n, d.data());
  if (m.eta > 0) {
    const double a1 = 1.0 / m.n, b1 = -std::log2(m.eta) / m.n;
    const double a2 = (a1 - 1.0) * kRootPerUnit, b2 = (std::log2(m.K) + b1 + kRootSpan) * kRootPerUnit - 0.5;
    for (int i = 0; i < kRootIv; ++i) {
      const double ai = d[2 * i], bi = d[2 * i + 1];
      d[2 * i] = b1 + ai + bi * b2;
      d[2 * i + 1] = a1 + bi * a2;
    }
  }
  root_table(m.nt, d.data() + kRootTabLen);
  return std::vector<T>(d.begin(), d.end());
}

template <typename T>
rve_status upload_root_tab(rve_s* h) {
  const std::vector<T> t = root_tables<T>(h->mat);
  if (!h->root_tab) {
    rve_status s = dalloc(h, &h->root_tab, (size_t)kRootTabs * sizeof(T));
    if (s) return s;
  }
  RVE_CUDA(h, cudaMemcpyAsync(h->root_tab, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

template <typename T>
XArgs<T> x_args(rve_s* h, const void* in, void* out, int it) {
  XArgs<T> a{};
  a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.H = h->H; a.L = h->L; a.xs = h->xs;
  a.nvox = h->nvox;
  a.dx = h->dx;
  a.tw = (const C2<T>*)h->tw_x;
  a.spec_in = (const C2<T>*)in;
  a.spec_out = (C2<T>*)out;
  a.ep = (T*)h->ep; a.v = (T*)h->v; a.al = (T*)h->al; a.eps_n = (T*)h->eps_n; a.sig_n = (T*)h->sig_n;
  a.grain = h->grain;
  a.Rg = (const T*)h->Rg;
  a.flow = h->flow;
  a.k.root_tab = (const T*)h->root_tab;
  a.k.M = make_mat<T>(h);
  if (h->lin_mode) {
    a.lin_B = (const T*)h->lin_B;
    a.lin_g = (const T*)h->lin_g;
    if (!out) a.eps_n = (T*)h->lin_mu;  // the linear-law commit writes the solution field here
  }
  // mixed load
  double M0[36];
  c0_mandel(h->lam0, h->mu0, M0);
  LoadDev& ld = a.k.ld;
  std::memset(&ld, 0, sizeof(ld));
  int fi[6], nf = 0;
  for (int c = 0; c < 6; ++c) {
    ld.free_mask[c] = h->ctrl[c] ? 0 : 1;
    ld.Sigma_m[c] = h->lin_mode ? 0.0 : h->Sigma[c] * kMw[c];
    if (!h->ctrl[c]) fi[nf++] = c;
  }
  ld.any_free = nf > 0;
  ld.s_ref = h->lin_mode ? h->lin_sref : 0.0;
  if (nf > 0) {
    std::vector<double> Mff(nf * nf);
    for (int i = 0; i < nf; ++i)
      for (int j = 0; j < nf; ++j) Mff[i * nf + j] = M0[fi[i] * 6 + fi[j]];
    invert(Mff.data(), nf);
    for (int i = 0; i < nf; ++i)
      for (int j = 0; j < nf; ++j) ld.Minv[fi[i] * 6 + fi[j]] = Mff[i * nf + j];
  }
  a.k.dt = (T)h->dt;
  a.k.nsub = h->opt.n_sub > 0 ? h->opt.n_sub : default_nsub(h->dt);
  a.partial = h->partial;
  a.counter = h->counter;
  a.st = h->st;
  a.it = it;
  a.done = out ? &h->st->done : nullptr;  // the commit (no output spectrum) always runs
  return a;
}

template <typename T>
LineArgs<T> y_args(rve_s* h, void* spec) {
  LineArgs<T> a{};
  a.d = h->dy;
  a.tw = (const C2<T>*)h->tw_y;
  a.spec = (C2<T>*)spec;
  a.H = h->H;
  a.HC = h->yHC;
  // component-interleaved spectra: CTA (kx chunk, kz) transforms all 6 components
  a.NC = 6;
  a.hstride = 6;
  a.n_o2 = 1;
  a.stride = (long long)h->H * 6;
  a.A = (long long)h->ny * h->H * 6;
  a.B = 0;
  a.done = &h->st->done;
  return a;
}

template <typename T>
ZArgs<T> z_args(rve_s* h, void* spec, const void* Pp, void* Po, int it) {
  ZArgs<T> a{};
  a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.H = h->H; a.HC = h->zHC;
  a.nvox = h->nvox;
  a.dz = h->dz;
  a.tw = (const C2<T>*)h->tw_z;
  a.spec = (C2<T>*)spec;
  a.P_prev = (const C2<T>*)Pp;
  a.P_out = (C2<T>*)Po;
  a.kx = (const T*)h->kx;
  a.ky = (const T*)h->ky;
  a.kzt = (const T*)h->kz;
  a.scheme = h->opt.green;
  a.lam0 = (T)h->lam0;
  a.mu0 = (T)h->mu0;
  a.invN = (T)(1.0 / (double)h->nvox);
  a.conv.tol = h->opt.tol;
  a.conv.fixed_iters = h->opt.fixed_iters;
  a.conv.max_iter = h->opt.max_iter > 0 ? h->opt.max_iter : 1000;
  a.conv.hist = h->dhist;
  a.conv.s_ref = h->lin_mode ? h->lin_sref : 0.0;
  a.done = &h->st->done;
  a.partial = h->partial;
  a.counter = h->counter;
  a.st = h->st;
  a.it = it;
  return a;
}

double vm_of(const double* s) {
  const double p = (s[0] + s[1] + s[2]) / 3.0;
  const double a = s[0] - p, b = s[1] - p, c = s[2] - p;
  return std::sqrt(1.5 * (a * a + b * b + c * c + 2.0 * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5])));
}

// Macroscopic increment and initial guess (first increment: C0-consistent free
// components; later ones: the previous increment's macroscopic step).
void initial_increment(rve_s* h, double dE0[6]) {
  int fi[6], ci[6], nf = 0, nc = 0;
  for (int c = 0; c < 6; ++c) (h->ctrl[c] ? ci[nc++] : fi[nf++]) = c;
  if (h->increment == 0) {
    double dm[6] = {0};
    for (int c = 0; c < 6; ++c) dm[c] = h->ctrl[c] ? h->Edot[c] * h->dt * kMw[c] : 0.0;
    if (nf > 0) {
      double M0[36];
      c0_mandel(h->lam0, h->mu0, M0);
      std::vector<double> Mff(nf * nf);
      for (int i = 0; i < nf; ++i)
        for (int j = 0; j < nf; ++j) Mff[i * nf + j] = M0[fi[i] * 6 + fi[j]];
      invert(Mff.data(), nf);
      double rhs[6] = {0};
      for (int i = 0; i < nf; ++i)
        for (int j = 0; j < nc; ++j) rhs[i] += M0[fi[i] * 6 + ci[j]] * dm[ci[j]];
      for (int i = 0; i < nf; ++i) {
        double x = 0.0;
        for (int j = 0; j < nf; ++j) x += Mff[i * nf + j] * rhs[j];
        dm[fi[i]] = -x;
      }
    }
    for (int c = 0; c < 6; ++c) dE0[c] = dm[c] / kMw[c];
  } else {
    for (int c = 0; c < 6; ++c) dE0[c] = h->ctrl[c] ? h->Edot[c] * h->dt : h->E_n[c] - h->E_prev[c];
  }
}

// Buffer rotation: iteration it reads strain spectrum S_in(it) and writes S_out(it)
// (then transformed in place); S_in(0) is the committed spectrum, S_out alternates
// between the two others, and S_in(it) = S_out(it - 1).  The tau_hat spectra rotate
// the same way.  The committed pair is only read, so a failed increment keeps it.
struct Rotation {
  int s0, s1, s2, p0, p1, p2;
  explicit Rotation(const rve_s* h)
      : s0(h->sb), s1((h->sb + 1) % 3), s2((h->sb + 2) % 3), p0(h->pb), p1((h->pb + 1) % 3), p2((h->pb + 2) % 3) {}
  int s_out(int it) const { return (it % 2 == 0) ? s1 : s2; }
  int s_in(int it) const { return it == 0 ? s0 : s_out(it - 1); }
  int p_out(int it) const { return (it % 2 == 0) ? p1 : p2; }
  int p_in(int it) const { return it == 0 ? p0 : p_out(it - 1); }
};

int max_iter_of(const rve_s* h) { return h->opt.max_iter > 0 ? h->opt.max_iter : 1000; }

int np_of(const rve_s* h) {
  const rve_material& m = h->mat;
  return h->lin_mode ? kLinearLaw : rate_variant(m.eta, m.K, m.Kt, is_small_int(m.n), is_small_int(m.nt));
}

// One fixed-point iteration (x pass, forward y, z + Green, inverse y) on stream s:
// strain spectrum si -> so, tau_hat spectra pi -> po.  it < 0: the kernels take the
// iteration index from the device (graph mode) and the residual kernel clears `cond`
// once it decides.  `slot` >= 0 brackets the launches with timing events.
template <typename T>
rve_status enqueue_one(rve_s* h, cudaStream_t s, int it, int si, int so, int pi, int po,
                       const cudaGraphConditionalHandle* cond, int slot) {
  const int np = np_of(h);
  const int zgrid_x = (h->H + h->zHC - 1) / h->zHC;
  const int ygrid_x = (h->H + h->yHC - 1) / h->yHC;
  const bool timed = slot >= 0;
  XArgs<T> xa = x_args<T>(h, h->spec[si], h->spec[so], it);
  if (timed) tstart(h, 4 * slot + 0, RVE_K_XPASS);
  RVE_CUDA(h, launch_xpass<T>(xa, np, false, h->xgrid, xsmem_total(h), s));
  if (timed) tstop(h, 4 * slot + 0);
  LineArgs<T> ya = y_args<T>(h, h->spec[so]);
  if (timed) tstart(h, 4 * slot + 1, RVE_K_YFWD);
  RVE_CUDA(h, launch_line<T>(ya, -1, dim3(ygrid_x, h->nz), h->ysmem, s));
  if (timed) tstop(h, 4 * slot + 1);
  ZArgs<T> za = z_args<T>(h, h->spec[so], h->P[pi], h->P[po], it);
  if (cond) {
    za.has_cond = 1;
    za.cond = *cond;
  }
  if (timed) tstart(h, 4 * slot + 2, RVE_K_ZGREEN);
  RVE_CUDA(h, launch_zgreen<T>(za, dim3(zgrid_x, h->ny), h->zsmem, s));
  if (timed) tstop(h, 4 * slot + 2);
  if (timed) tstart(h, 4 * slot + 3, RVE_K_YINV);
  RVE_CUDA(h, launch_line<T>(ya, +1, dim3(ygrid_x, h->nz), h->ysmem, s));
  if (timed) tstop(h, 4 * slot + 3);
  return RVE_OK;
}

// Enqueues iterations inc_it0 .. inc_it0 + inc_nb - 1, then the status copy and ev_sync.
// The residual kernel decides convergence on the device; later launches of the batch
// return at once.
template <typename T>
rve_status enqueue_iterations(rve_s* h) {
  cudaStream_t s = h->stream;
  const Rotation r(h);
  h->inc_nb = std::min(kBatch, max_iter_of(h) - h->inc_it0);
  for (int b = 0; b < h->inc_nb; ++b) {
    const int it = h->inc_it0 + b;
    rve_status st = enqueue_one<T>(h, s, it, r.s_in(it), r.s_out(it), r.p_in(it), r.p_out(it), nullptr, b);
    if (st) return st;
  }
  RVE_CUDA(h, cudaMemcpyAsync(h->st_host, h->st, sizeof(IterStatus), cudaMemcpyDeviceToHost, s));
  RVE_CUDA(h, cudaEventRecord(h->ev_sync, s));
  return RVE_OK;
}

bool use_graphs(const rve_s* h) { return h->opt.graphs && !h->opt.timing; }

// Graph of one increment for the current buffer rotation (h->sb): iteration 0
// (S0 -> S1), then a while-node whose body runs two iterations (S1 -> S2, S2 -> S1) and a
// guard kernel, then the commit (a no-op unless the increment converged; it reads the
// converged iteration's spectrum) and the status copy to the host.  The loop ends when the
// residual kernel decides (converged, NaN, or the iteration cap) or, independently, after
// max_iter / 2 + 2 body executions.
template <typename T>
rve_status build_graph(rve_s* h) {
  const int key = h->sb;
  const Rotation r(h);
  for (int k = 0; k < 2; ++k)
    if (!h->cap[k]) RVE_CUDA(h, cudaStreamCreateWithFlags(&h->cap[k], cudaStreamNonBlocking));
  cudaStream_t cs = h->cap[0], cb = h->cap[1];
  cudaGraph_t g = nullptr;
  RVE_CUDA(h, cudaGraphCreate(&g, 0));
  h->graph[key] = g;  // destroyed by drop_graphs
  cudaGraphConditionalHandle cond;
  RVE_CUDA(h, cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault));
  RVE_CUDA(h, cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  rve_status st = RVE_OK;
  cudaError_t e = cudaSuccess;
  bool body_open = false;
  do {
    if ((st = enqueue_one<T>(h, cs, -1, r.s0, r.s1, r.p0, r.p1, &cond, -1))) break;
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &nd)) != cudaSuccess) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wn;
    if ((e = cudaGraphAddNode(&wn, g, deps, nullptr, nd, &cp)) != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamUpdateCaptureDependencies(cs, &wn, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess)
      break;
    if ((e = cudaStreamBeginCaptureToGraph(cb, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
      break;
    body_open = true;
    if ((st = enqueue_one<T>(h, cb, -1, r.s1, r.s2, r.p1, r.p2, &cond, -1))) break;
    if ((st = enqueue_one<T>(h, cb, -1, r.s2, r.s1, r.p2, r.p1, &cond, -1))) break;
    if ((e = launch_loop_guard<T>(h->st, max_iter_of(h) / 2 + 2, cond, cb)) != cudaSuccess) break;
    cudaGraph_t bout = nullptr;
    body_open = false;
    if ((e = cudaStreamEndCapture(cb, &bout)) != cudaSuccess) break;
    XArgs<T> ca = x_args<T>(h, h->spec[r.s0], nullptr, -1);
    ca.pick = 1;
    ca.cand[0] = (const C2<T>*)h->spec[r.s0];
    ca.cand[1] = (const C2<T>*)h->spec[r.s1];
    ca.cand[2] = (const C2<T>*)h->spec[r.s2];
    if ((e = launch_xpass<T>(ca, np_of(h), true, h->xgrid, xsmem_total(h), cs)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(h->st_host, h->st, sizeof(IterStatus), cudaMemcpyDeviceToHost, cs)) != cudaSuccess) break;
  } while (false);
  if (body_open) {
    cudaGraph_t tmp = nullptr;
    cudaStreamEndCapture(cb, &tmp);
  }
  cudaGraph_t out = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cs, &out);
  if (st == RVE_OK && e != cudaSuccess) st = cuda_fail(h, e, "graph capture");
  if (st == RVE_OK && e2 != cudaSuccess) st = cuda_fail(h, e2, "cudaStreamEndCapture");
  if (st == RVE_OK) {
    e = cudaGraphInstantiate(&h->gexec[key], g, 0);
    if (e != cudaSuccess) st = cuda_fail(h, e, "cudaGraphInstantiate");
  }
  if (st != RVE_OK) {
    cudaGetLastError();
    drop_graphs(h);
  }
  return st;
}

// FFT tile autotuner: times the y and z passes for kx tile widths 1, 2, 4, 8, 16 on scratch
// buffers (a non-committed strain spectrum, the non-committed tau_hat spectra, a scratch
// status record) and keeps the fastest.  No result depends on the widths: every
// sequence's FFT is the same arithmetic, and the residual is summed per (ky, kx) column.
template <typename T>
rve_status tune_tiles(rve_s* h) {
  h->tuned = true;
  const bool ty = h->opt.y_tile <= 0, tz = h->opt.z_tile <= 0;
  if (!ty && !tz) return RVE_OK;
  cudaStream_t s = h->stream;
  int smax = 0;
  RVE_CUDA(h, cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->opt.device));
  void* sp = h->spec[(h->sb + 1) % 3];
  void* pp = h->P[(h->pb + 1) % 3];
  void* po = h->P[(h->pb + 2) % 3];
  const size_t spec_bytes = (size_t)6 * h->NL * h->H * 2 * sizeof(T);
  RVE_CUDA(h, cudaMemsetAsync(sp, 0, spec_bytes, s));
  RVE_CUDA(h, cudaMemsetAsync(pp, 0, spec_bytes, s));
  RVE_CUDA(h, cudaMemsetAsync(h->st_tune, 0, sizeof(IterStatus), s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RVE_CUDA(h, cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(h, e, "cudaEventCreate");
  }
  // 1 warm-up launch, then 3 timed
  auto timed = [&](auto launch, float* ms) -> cudaError_t {
    cudaError_t r = launch();
    if (r == cudaSuccess) r = cudaEventRecord(e0, s);
    for (int k = 0; k < 3 && r == cudaSuccess; ++k) r = launch();
    if (r == cudaSuccess) r = cudaEventRecord(e1, s);
    if (r == cudaSuccess) r = cudaEventSynchronize(e1);
    if (r == cudaSuccess) r = cudaEventElapsedTime(ms, e0, e1);
    return r;
  };
  const int cands[5] = {1, 2, 4, 8, 16};
  if (ty) {
    float best = 1e30f;
    int bhc = h->yHC;
    int prev = 0;
    for (int c : cands) {
      const int pm = pencil_max_hc(h->ny);
      const int hc = std::min(std::min(c, h->H), pm > 0 ? pm : c);
      if (hc == prev) continue;  // same as the previous width
      prev = hc;
      const size_t sm = y_smem<T>(h, hc);
      if (sm > (size_t)smax) continue;
      LineArgs<T> ya = y_args<T>(h, sp);
      ya.HC = hc;
      ya.done = nullptr;
      const dim3 grid((h->H + hc - 1) / hc, h->nz);
      float ms = 0.f;
      e = timed([&] { return launch_line<T>(ya, -1, grid, sm, s); }, &ms);
      if (e != cudaSuccess) break;
      if (ms < best) {
        best = ms;
        bhc = hc;
      }
    }
    h->yHC = bhc;
    h->ysmem = y_smem<T>(h, bhc);
  }
  if (e == cudaSuccess && tz) {
    float best = 1e30f;
    int bhc = h->zHC;
    int prev = 0;
    for (int c : cands) {
      const int pm = pencil_max_hc(h->nz);
      const int hc = std::min(std::min(c, h->H), pm > 0 ? pm : c);
      if (hc == prev) continue;
      prev = hc;
      const size_t sm = z_smem<T>(h, hc);
      if (sm > (size_t)smax) continue;
      ZArgs<T> za = z_args<T>(h, sp, pp, po, 0);
      za.HC = hc;
      za.st = h->st_tune;
      za.done = &h->st_tune->done;
      za.conv.hist = h->hist_tune;
      za.conv.fixed_iters = 1 << 30;  // never decides
      za.conv.max_iter = 1 << 30;
      za.has_cond = 0;
      const dim3 grid((h->H + hc - 1) / hc, h->ny);
      float ms = 0.f;
      e = timed([&] { return launch_zgreen<T>(za, grid, sm, s); }, &ms);
      if (e != cudaSuccess) break;
      if (ms < best) {
        best = ms;
        bhc = hc;
      }
    }
    h->zHC = bhc;
    h->zsmem = z_smem<T>(h, bhc);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(h, e, "tile autotuner");
  return RVE_OK;
}

// Starts increment n -> n+1: macroscopic step and initial guess (a1), then the first
// batch of iterations (or the whole increment as one graph launch).
template <typename T>
rve_status inc_prepare(rve_s* h) {
  cudaStream_t s = h->stream;
  if (h->opt.autotune && !h->tuned) {
    rve_status st = tune_tiles<T>(h);
    if (st) return st;
  }
  initial_increment(h, h->inc_dE0);
  // E^(0) into slot 0 of the device status record; clear the NaN flag, the decision and
  // the device-side iteration counters
  for (int c = 0; c < 6; ++c) h->st_host->E[0][c] = h->E_n[c] + h->inc_dE0[c];
  RVE_CUDA(h, cudaMemcpyAsync(h->st->E[0], h->st_host->E[0], 6 * sizeof(double), cudaMemcpyHostToDevice, s));
  RVE_CUDA(h, cudaMemsetAsync(&h->st->nan_flag, 0, 5 * sizeof(int), s));
  const Rotation r(h);
  tstart(h, kSlotShift, RVE_K_SHIFT);
  RVE_CUDA(h, launch_shift<T>((C2<T>*)h->spec[r.s0], (C2<T>*)h->backup, h->NL, h->H, h->inc_dE0, false, s));
  tstop(h, kSlotShift);
  return RVE_OK;
}

template <typename T>
rve_status inc_begin(rve_s* h) {
  cudaStream_t s = h->stream;
  rve_status pst = inc_prepare<T>(h);
  if (pst) return pst;
  if (use_graphs(h)) {
    if (!h->gexec[h->sb]) {
      rve_status st = build_graph<T>(h);
      if (st) return st;
    }
    RVE_CUDA(h, cudaGraphLaunch(h->gexec[h->sb], s));
    RVE_CUDA(h, cudaEventRecord(h->ev_sync, s));
    h->inc_phase = 3;
    return RVE_OK;
  }
  h->inc_it0 = 0;
  h->inc_phase = 1;
  rve_status st = enqueue_iterations<T>(h);
  if (st) h->inc_phase = 0;
  return st;
}

// The increment's iterations are over (status in st_host): fetch the residual history and,
// unless it converged, roll the start-of-increment shift back and report.
template <typename T>
rve_status close_iterations(rve_s* h, const IterStatus& stat) {
  cudaStream_t s = h->stream;
  const Rotation r(h);
  const int max_iter = max_iter_of(h);
  const int last = stat.done ? stat.done_it : std::max(0, std::min(stat.it_dev, max_iter) - 1);
  std::vector<double> hh(2 * (size_t)(last + 1));
  RVE_CUDA(h, cudaMemcpyAsync(hh.data(), h->dhist, hh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  RVE_CUDA(h, cudaStreamSynchronize(s));
  h->res_e.resize(last + 1);
  h->res_c.resize(last + 1);
  for (int i = 0; i <= last; ++i) {
    h->res_e[i] = hh[2 * i];
    h->res_c[i] = hh[2 * i + 1];
  }
  if (stat.done == 1) return RVE_OK;
  RVE_CUDA(h, launch_shift<T>((C2<T>*)h->spec[r.s0], (C2<T>*)h->backup, h->NL, h->H, h->inc_dE0, true, s));
  RVE_CUDA(h, cudaStreamSynchronize(s));
  if (stat.done == 2)
    return fail(h, RVE_ERR_NAN, std::string("NaN or Inf in the ") +
                                    ((stat.nan_flag & 1) ? "mean stress" : "equilibrium residual") + " at increment " +
                                    std::to_string(h->increment + 1) + ", iteration " + std::to_string(last));
  if (stat.done == 0)
    return fail(h, RVE_ERR_STATE, "increment " + std::to_string(h->increment + 1) +
                                      ": the device loop ended without a decision");
  char buf[200];
  std::snprintf(buf, sizeof(buf), "increment %d: no convergence in %d iterations (e=%.3e, cF=%.3e)",
                h->increment + 1, max_iter, stat.e_eq, stat.cF);
  return fail(h, RVE_ERR_NOT_CONVERGED, buf);
}

// The commit completed (status in st_host): advance the host state and record the
// increment's effective results.
rve_status finish_increment(rve_s* h, long long* iters) {
  const Rotation r(h);
  const int it = h->inc_last;
  h->sb = r.s_in(it);
  h->pb = r.p_in(it);
  for (int c = 0; c < 6; ++c) {
    h->E_prev[c] = h->E_n[c];
    h->E_n[c] = h->inc_E[c];
  }
  h->time += h->dt;
  h->increment += 1;
  rve_effective rec;
  std::memset(&rec, 0, sizeof(rec));
  rec.increment = h->increment;
  rec.iterations = it + 1;
  rec.time = h->time;
  for (int c = 0; c < 6; ++c) {
    rec.E[c] = h->inc_E[c];
    rec.S[c] = h->st_host->sig_mean[c];
  }
  rec.S_eq_of_mean = vm_of(rec.S);
  rec.mean_S_eq = h->st_host->eff[0];
  rec.mean_f = h->st_host->eff[1];
  rec.mean_v = h->st_host->eff[2];
  rec.residual = h->inc_e;
  rec.stress_residual = h->inc_c;
  h->hist.push_back(rec);
  if (iters) *iters += it + 1;
  if (h->st_host->nan_flag) return fail(h, RVE_ERR_NAN, "NaN or Inf in the committed fields");
  return RVE_OK;
}

void note_converged(rve_s* h, const IterStatus& stat) {
  const int it = stat.done_it;
  h->inc_last = it;
  h->inc_e = stat.e_eq;
  h->inc_c = stat.cF;
  for (int c = 0; c < 6; ++c) h->inc_E[c] = stat.E[it & 1][c];
}

// Resumes after ev_sync completed.  Sets *finished when the increment is committed (or
// has failed and been rolled back; the status says which).
template <typename T>
rve_status inc_advance(rve_s* h, bool* finished, long long* iters) {
  cudaStream_t s = h->stream;
  const Rotation r(h);
  *finished = true;
  const int phase = h->inc_phase;
  h->inc_phase = 0;
  if (phase == 3) {  // the whole increment ran as one graph (the commit included)
    const IterStatus stat = *h->st_host;
    rve_status st = close_iterations<T>(h, stat);
    if (st) return st;
    note_converged(h, stat);
    return finish_increment(h, iters);
  }
  if (phase == 1) {
    const int done = h->st_host->done;
    const int it0 = h->inc_it0, nb = h->inc_nb;
    tcollect(h, done ? h->st_host->done_it - it0 + 1 : nb);
    if (!done && it0 + nb < max_iter_of(h)) {
      h->inc_it0 += nb;
      h->inc_phase = 1;
      *finished = false;
      rve_status st = enqueue_iterations<T>(h);
      if (st) { h->inc_phase = 0; *finished = true; }
      return st;
    }
    const IterStatus stat = *h->st_host;
    rve_status st = close_iterations<T>(h, stat);
    if (st) return st;
    // commit the converged iterate
    note_converged(h, stat);
    const int it = stat.done_it;
    XArgs<T> ca = x_args<T>(h, h->spec[r.s_in(it)], nullptr, it);
    tstart(h, kSlotCommit, RVE_K_COMMIT);
    RVE_CUDA(h, launch_xpass<T>(ca, np_of(h), true, h->xgrid, xsmem_total(h), s));
    tstop(h, kSlotCommit);
    RVE_CUDA(h, cudaMemcpyAsync(h->st_host, h->st, sizeof(IterStatus), cudaMemcpyDeviceToHost, s));
    RVE_CUDA(h, cudaEventRecord(h->ev_sync, s));
    h->inc_phase = 2;
    *finished = false;
    return RVE_OK;
  }
  if (phase != 2) return fail(h, RVE_ERR_STATE, "no increment in progress");
  // the commit completed
  tcollect(h, 0);
  return finish_increment(h, iters);
}

rve_status inc_begin_any(rve_s* h) {
  return h->opt.precision == RVE_FP64 ? inc_begin<double>(h) : inc_begin<float>(h);
}

rve_status inc_advance_any(rve_s* h, bool* finished, long long* iters) {
  return h->opt.precision == RVE_FP64 ? inc_advance<double>(h, finished, iters)
                                      : inc_advance<float>(h, finished, iters);
}

// One increment on the handle's stream, waiting for each phase.
rve_status step_one(rve_s* h, long long* iters) {
  NvtxRange range("rve increment");
  rve_status st = inc_begin_any(h);
  bool finished = st != RVE_OK;
  while (!finished) {
    cudaError_t e = cudaEventSynchronize(h->ev_sync);
    if (e != cudaSuccess) {
      h->inc_phase = 0;
      return cuda_fail(h, e, "cudaEventSynchronize");
    }
    st = inc_advance_any(h, &finished, iters);
  }
  return st;
}

// ---------------------------------------------------------------- grouped batch ------
// An ensemble stepped as one group (rve_step_batch): every pass of a fixed-point iteration
// is one launch over all members (k_*_group; each CTA runs its member's pass exactly as the
// member's own launch would), the members iterate in lockstep (a member whose increment is
// decided returns at once from later launches), and one increment of the whole group is
// one CUDA graph launch: iteration 0, a while-node whose body runs two iterations and the
// group guard, the commit, and every member's status copy.

int nsub_of(const rve_s* h) { return h->opt.n_sub > 0 ? h->opt.n_sub : default_nsub(h->dt); }

// Handles that can run as one group: one device and precision, the graph loop, the same
// material, load and substeps (the grouped x pass reads them once), at most kMaxGroup.
bool groupable(rve_s* const* hs, int n) {
  if (n < 2 || n > kMaxGroup) return false;
  const rve_s* a = hs[0];
  for (int i = 0; i < n; ++i) {
    const rve_s* h = hs[i];
    if (!h->opt.batch_group || !use_graphs(h) || h->lin_mode || h->opt.precision != a->opt.precision ||
        h->opt.device != a->opt.device)
      return false;
    if (std::memcmp(&h->mat, &a->mat, sizeof(rve_material)) != 0 || h->dt != a->dt || nsub_of(h) != nsub_of(a))
      return false;
    for (int c = 0; c < 6; ++c)
      if (h->Edot[c] != a->Edot[c] || h->ctrl[c] != a->ctrl[c] || h->Sigma[c] != a->Sigma[c]) return false;
  }
  return true;
}

// Arguments of one grouped iteration (heap: the blocks are kilobytes each).
template <typename T>
struct GroupIter {
  XGroup<T> x;
  LineGroup<T> y;
  ZGroup<T> z;
  int xgrid = 0, ygrid = 0, zgrid = 0;
  size_t xsmem = 0, ysmem = 0, zsmem = 0;
};

// which: 0 = iteration 0 (S0 -> S1), 1 = first body iteration (S1 -> S2), 2 = second (S2 -> S1).
template <typename T>
void group_iter_args(const std::vector<rve_s*>& hs, int which, GroupIter<T>& g) {
  const int n = (int)hs.size();
  for (int m = 0; m < n; ++m) {
    rve_s* h = hs[m];
    const Rotation r(h);
    const int si = which == 0 ? r.s0 : (which == 1 ? r.s1 : r.s2);
    const int so = which == 1 ? r.s2 : r.s1;
    const int pi = which == 0 ? r.p0 : (which == 1 ? r.p1 : r.p2);
    const int po = which == 1 ? r.p2 : r.p1;
    g.x.m[m] = x_args<T>(h, h->spec[si], h->spec[so], -1);
    g.x.start[m] = g.xgrid;
    g.x.gx[m] = h->xgrid;
    g.xgrid += h->xgrid;
    g.xsmem = std::max(g.xsmem, xsmem_total(h));
    g.y.m[m] = y_args<T>(h, h->spec[so]);
    const int ygx = (h->H + h->yHC - 1) / h->yHC;
    g.y.start[m] = g.ygrid;
    g.y.gx[m] = ygx;
    g.ygrid += ygx * h->nz;
    g.ysmem = std::max(g.ysmem, line_group_smem<T>(h->ny, h->yHC));
    ZArgs<T> za = z_args<T>(h, h->spec[so], h->P[pi], h->P[po], -1);
    za.has_cond = 0;  // the group guard ends the loop
    g.z.m[m] = za;
    const int zgx = (h->H + h->zHC - 1) / h->zHC;
    g.z.start[m] = g.zgrid;
    g.z.gx[m] = zgx;
    g.zgrid += zgx * h->ny;
    g.zsmem = std::max(g.zsmem, zgreen_group_smem<T>(h->nz, h->zHC));
  }
  g.x.k = g.x.m[0].k;
  g.x.n = g.y.n = g.z.n = n;
  g.x.start[n] = g.xgrid;
  g.y.start[n] = g.ygrid;
  g.z.start[n] = g.zgrid;
}

template <typename T>
cudaError_t group_iteration(const GroupIter<T>& g, int np, cudaStream_t s) {
  cudaError_t e = launch_xpass_group<T>(g.x, np, false, g.xgrid, g.xsmem, s);
  if (e == cudaSuccess) e = launch_line_group<T>(g.y, -1, g.ygrid, g.ysmem, s);
  if (e == cudaSuccess) e = launch_zgreen_group<T>(g.z, g.zgrid, g.zsmem, s);
  if (e == cudaSuccess) e = launch_line_group<T>(g.y, +1, g.ygrid, g.ysmem, s);
  return e;
}

struct GroupGraph {
  std::vector<int> key;  // (index, sb, pb) of every member: the buffer rotations baked in
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

void drop_group_graph(GroupGraph& gg) {
  if (gg.exec) cudaGraphExecDestroy(gg.exec);
  if (gg.graph) cudaGraphDestroy(gg.graph);
  gg.exec = nullptr;
  gg.graph = nullptr;
}

// The graph of one increment of the group (see above), captured on cs (main graph) and cb
// (loop body).
template <typename T>
cudaError_t build_group_graph(const std::vector<rve_s*>& hs, cudaStream_t cs, cudaStream_t cb, GroupGraph& out) {
  const int n = (int)hs.size();
  const int np = np_of(hs[0]);
  auto it0 = std::make_unique<GroupIter<T>>();
  auto itA = std::make_unique<GroupIter<T>>();
  auto itB = std::make_unique<GroupIter<T>>();
  auto cm = std::make_unique<XGroup<T>>();
  group_iter_args<T>(hs, 0, *it0);
  group_iter_args<T>(hs, 1, *itA);
  group_iter_args<T>(hs, 2, *itB);
  GuardGroup gd{};
  gd.n = n;
  gd.limit = 0;
  int cgrid = 0;
  size_t csmem = 0;
  for (int m = 0; m < n; ++m) {
    rve_s* h = hs[m];
    const Rotation r(h);
    gd.st[m] = h->st;
    gd.limit = std::max(gd.limit, max_iter_of(h) / 2 + 2);
    XArgs<T> ca = x_args<T>(h, h->spec[r.s0], nullptr, -1);
    ca.pick = 1;
    ca.cand[0] = (const C2<T>*)h->spec[r.s0];
    ca.cand[1] = (const C2<T>*)h->spec[r.s1];
    ca.cand[2] = (const C2<T>*)h->spec[r.s2];
    cm->m[m] = ca;
    cm->start[m] = cgrid;
    cm->gx[m] = h->xgrid;
    cgrid += h->xgrid;
    csmem = std::max(csmem, xsmem_total(h));
  }
  cm->k = cm->m[0].k;
  cm->n = n;
  cm->start[n] = cgrid;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  out.graph = g;
  cudaGraphConditionalHandle cond;
  if ((e = cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
  if ((e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
    return e;
  bool body_open = false;
  do {
    if ((e = group_iteration<T>(*it0, np, cs)) != cudaSuccess) break;
    if ((e = launch_group_guard<T>(gd, cond, cs)) != cudaSuccess) break;
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &nd)) != cudaSuccess) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wn;
    if ((e = cudaGraphAddNode(&wn, g, deps, nullptr, nd, &cp)) != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamUpdateCaptureDependencies(cs, &wn, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess)
      break;
    if ((e = cudaStreamBeginCaptureToGraph(cb, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
      break;
    body_open = true;
    if ((e = group_iteration<T>(*itA, np, cb)) != cudaSuccess) break;
    if ((e = group_iteration<T>(*itB, np, cb)) != cudaSuccess) break;
    if ((e = launch_group_guard<T>(gd, cond, cb)) != cudaSuccess) break;
    cudaGraph_t bout = nullptr;
    body_open = false;
    if ((e = cudaStreamEndCapture(cb, &bout)) != cudaSuccess) break;
    if ((e = launch_xpass_group<T>(*cm, np, true, cgrid, csmem, cs)) != cudaSuccess) break;
    for (int m = 0; m < n && e == cudaSuccess; ++m)
      e = cudaMemcpyAsync(hs[m]->st_host, hs[m]->st, sizeof(IterStatus), cudaMemcpyDeviceToHost, cs);
  } while (false);
  if (body_open) {
    cudaGraph_t tmp = nullptr;
    cudaStreamEndCapture(cb, &tmp);
  }
  cudaGraph_t done = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cs, &done);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&out.exec, g, 0);
  return e;
}

// rve_step_batch for a groupable batch: n_increments increments of every member as one
// group on a private stream (ordered after each member's own stream and before later work
// there).  A failing member keeps its last committed increment and leaves the group.
template <typename T>
rve_status step_batch_group(rve_s* const* hs, int n, int n_increments, long long* iters, int* failed) {
  rve_status first = RVE_OK;
  int first_i = -1;
  auto note = [&](int i, rve_status st) {
    if (st != RVE_OK && first == RVE_OK) {
      first = st;
      first_i = i;
    }
  };
  cudaStream_t gs = nullptr, cap[2] = {nullptr, nullptr};
  cudaError_t e = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&cap[k], cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    for (cudaStream_t q : {gs, cap[0], cap[1]})
      if (q) cudaStreamDestroy(q);
    return cuda_fail(nullptr, e, "group stream set-up");
  }
  std::vector<cudaStream_t> orig(n);
  for (int i = 0; i < n; ++i) {
    rve_s* h = hs[i];
    orig[i] = h->stream;
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_sync, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(gs, h->ev_sync, 0);
    h->stream = gs;
  }
  if (e != cudaSuccess) note(0, cuda_fail(hs[0], e, "group stream ordering"));
  std::vector<char> active(n, first == RVE_OK ? 1 : 0);
  std::vector<GroupGraph> cache;
  constexpr size_t kCache = 8;
  for (int inc = 0; inc < n_increments; ++inc) {
    std::vector<rve_s*> cur;
    std::vector<int> idx;
    for (int i = 0; i < n; ++i) {
      if (!active[i]) continue;
      rve_status st = inc_prepare<T>(hs[i]);
      if (st) {
        note(i, st);
        active[i] = 0;
        continue;
      }
      cur.push_back(hs[i]);
      idx.push_back(i);
    }
    if (cur.empty()) break;
    NvtxRange range("rve group increment");
    std::vector<int> key;
    for (size_t m = 0; m < cur.size(); ++m) key.insert(key.end(), {idx[m], cur[m]->sb, cur[m]->pb});
    GroupGraph* gg = nullptr;
    for (GroupGraph& c : cache)
      if (c.key == key) gg = &c;
    if (!gg) {
      if (cache.size() >= kCache) {
        drop_group_graph(cache.front());
        cache.erase(cache.begin());
      }
      cache.emplace_back();
      gg = &cache.back();
      gg->key = key;
      e = build_group_graph<T>(cur, cap[0], cap[1], *gg);
      if (e != cudaSuccess) {
        cudaGetLastError();
        drop_group_graph(*gg);
        cache.pop_back();
        for (int i : idx) active[i] = 0;
        note(idx[0], cuda_fail(cur[0], e, "group graph"));
        break;
      }
    }
    e = cudaGraphLaunch(gg->exec, gs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(gs);
    if (e != cudaSuccess) {
      for (int i : idx) active[i] = 0;
      note(idx[0], cuda_fail(cur[0], e, "group increment"));
      break;
    }
    for (size_t m = 0; m < cur.size(); ++m) {
      rve_s* h = cur[m];
      const IterStatus stat = *h->st_host;
      rve_status st = close_iterations<T>(h, stat);
      if (st == RVE_OK) {
        note_converged(h, stat);
        st = finish_increment(h, iters);
      }
      if (st) {
        note(idx[m], st);
        active[idx[m]] = 0;
      }
    }
  }
  for (GroupGraph& c : cache) drop_group_graph(c);
  for (int i = 0; i < n; ++i) {
    rve_s* h = hs[i];
    e = cudaEventRecord(h->ev_sync, gs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(orig[i], h->ev_sync, 0);
    if (e != cudaSuccess) note(i, cuda_fail(h, e, "group stream join"));
    h->stream = orig[i];
  }
  for (cudaStream_t q : {gs, cap[0], cap[1]}) cudaStreamDestroy(q);
  if (failed) *failed = first_i;
  if (first != RVE_OK) g_err = "handle " + std::to_string(first_i) + ": " + hs[first_i]->err;
  return first;
}

// ---------------------------------------------------------------- adjoint ------------
// Per-voxel scratch of the adjoint of one increment, in units of T per voxel.
enum AdjSlot {
  kAdjRvox = 0,                     // 9  rotations per voxel
  kAdjB = kAdjRvox + 9,             // 36 B of the linear law s = B mu - g
  kAdjG = kAdjB + 36,               // 6  g
  kAdjMu = kAdjG + 6,               // 6  adjoint solution mu
  kAdjSigB = kAdjMu + 6,            // 6  stress adjoint fed to the reverse pass
  kAdjStB = kAdjSigB + 6,           // 34 state adjoint (direct part)
  kAdjStZ = kAdjStB + 34,           // 34 state adjoint (constraint part / zero input)
  kAdjEbA = kAdjStZ + 34,           // 6  d/d eps, direct part
  kAdjEnA = kAdjEbA + 6,            // 6  d/d eps_prev, direct part
  kAdjEnB = kAdjEnA + 6,            // 6  d/d eps_prev, constraint part
  kAdjRbA = kAdjEnB + 6,            // 9
  kAdjRbB = kAdjRbA + 9,            // 9
  kAdjPbA = kAdjRbB + 9,            // 9
  kAdjPbB = kAdjPbA + 9,            // 9
  kAdjEpsP = kAdjPbB + 9,           // 6  strain at t_{n-1}
  kAdjEpsC = kAdjEpsP + 6,          // 6  strain at t_n
  kAdjStP = kAdjEpsC + 6,           // 34 state at t_{n-1}
  kAdjEbIn = kAdjStP + 34,          // 6  adjoint of the strain at t_n from the next increment
  kAdjJ = kAdjEbIn + 6,             // 36 tangent rows
  kAdjDummy = kAdjJ + 36,           // 30 unused outputs (eps_b 6, eps_n_b 6, R_b 9, param_b 9)
  kAdjTotal = kAdjDummy + 30
};

template <typename T>
rve_status adjoint_increment(rve_s* h, const double* eps_prev, const double* eps_cur, const double* state_prev,
                             const double dS[6], double dt_n, double* state_b, double* eps_b, double* pgrad,
                             double* egrad, long long* iters) {
  cudaStream_t s = h->stream;
  const long long n = h->nvox;
  const size_t N = (size_t)n;
  if (!h->adj) {
    rve_status st = dalloc(h, &h->adj, (size_t)kAdjTotal * N * sizeof(T));
    if (st) return st;
  }
  T* A = (T*)h->adj;
  auto at = [&](int slot) { return A + (size_t)slot * N; };
  const MatDev<T> M = make_mat<T>(h);
  const rve_material& m = h->mat;
  const int np = rate_variant(m.eta, m.K, m.Kt, is_small_int(m.n), is_small_int(m.nt));
  const int nsub = h->opt.n_sub > 0 ? h->opt.n_sub : default_nsub(dt_n);
  if (nsub > kMaxSubVjp) return fail(h, RVE_ERR_UNSUPPORTED, "adjoint: more than 16 RK4 substeps per increment");
  const T dt = (T)dt_n;
  const T* tab = (const T*)h->root_tab;
  // inputs in the working precision
  RVE_CUDA(h, launch_adj<T>(4, 6 * n, s, eps_prev, nullptr, nullptr, at(kAdjEpsP), nullptr, nullptr));
  RVE_CUDA(h, launch_adj<T>(4, 6 * n, s, eps_cur, nullptr, nullptr, at(kAdjEpsC), nullptr, nullptr));
  RVE_CUDA(h, launch_adj<T>(4, 34 * n, s, state_prev, nullptr, nullptr, at(kAdjStP), nullptr, nullptr));
  RVE_CUDA(h, launch_adj<T>(4, 34 * n, s, state_b, nullptr, nullptr, at(kAdjStB), nullptr, nullptr));
  RVE_CUDA(h, launch_adj<T>(4, 6 * n, s, eps_b, nullptr, nullptr, at(kAdjEbIn), nullptr, nullptr));
  RVE_CUDA(h, launch_adj<T>(0, n, s, h->grain, h->Rg, nullptr, at(kAdjRvox), nullptr, nullptr));
  // one stored forward pass per voxel, then the reverse sweeps: the tangent rows
  // d sigma_k / d eps and the direct part (stress adjoint dS / N everywhere, the state
  // adjoint from later increments)
  double v6[6];
  for (int c = 0; c < 6; ++c) v6[c] = dS[c] / (double)n;
  RVE_CUDA(h, launch_adj_tangent<T>(M, np, n, at(kAdjRvox), at(kAdjEpsP), at(kAdjEpsC), at(kAdjStP), dt, nsub, v6,
                                    at(kAdjStB), at(kAdjJ), at(kAdjEbA), at(kAdjEnA), at(kAdjRbA), at(kAdjPbA), tab,
                                    s));
  RVE_CUDA(h, launch_adj<T>(2, n, s, at(kAdjJ), at(kAdjEbA), at(kAdjEbIn), at(kAdjB), at(kAdjG), nullptr));
  // source scale |g|_rms = sqrt(<g : g>): per-block partial sums (into the unused-output
  // slot, free until the constraint part) added on the host in a fixed order
  double g_rms = 0.0;
  {
    const size_t nb = (N + 255) / 256;
    std::vector<double> part(nb);
    RVE_CUDA(h, launch_adj<T>(6, n, s, at(kAdjG), nullptr, nullptr, at(kAdjDummy), nullptr, nullptr));
    RVE_CUDA(h, cudaMemcpyAsync(part.data(), at(kAdjDummy), nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    RVE_CUDA(h, cudaStreamSynchronize(s));
    double q = 0.0;
    for (double x : part) q += x;
    if (!std::isfinite(q)) return fail(h, RVE_ERR_NAN, "adjoint: non-finite source");
    g_rms = std::sqrt(q / (double)n);
  }
  // adjoint fixed point: mu compatible with zero controlled macro components, s = B mu - g
  // equilibrated with zero mean on the free components (the forward iteration, linear law).
  // Its relative errors are taken against max(|<s>|, |g|_rms): the mean of s alone can
  // vanish (it does exactly when g = 0, e.g. an elastic increment without misfit).  With
  // g = 0 the solution is mu = 0 and no iteration runs.
  if (g_rms == 0.0) {
    RVE_CUDA(h, cudaMemsetAsync(at(kAdjMu), 0, 6 * N * sizeof(T), s));
  } else {
    const Rotation r(h);
    const size_t spec_bytes = (size_t)6 * h->NL * h->H * 2 * sizeof(T);
    RVE_CUDA(h, cudaMemsetAsync(h->spec[r.s0], 0, spec_bytes, s));
    RVE_CUDA(h, cudaMemsetAsync(h->P[r.p0], 0, spec_bytes, s));
    std::memset(h->st_host->E[0], 0, sizeof(h->st_host->E[0]));
    RVE_CUDA(h, cudaMemcpyAsync(h->st->E[0], h->st_host->E[0], 6 * sizeof(double), cudaMemcpyHostToDevice, s));
    RVE_CUDA(h, cudaMemsetAsync(&h->st->nan_flag, 0, 5 * sizeof(int), s));
    h->lin_mode = true;
    h->lin_sref = g_rms;
    h->lin_B = at(kAdjB);
    h->lin_g = at(kAdjG);
    h->lin_mu = at(kAdjMu);
    const int max_iter = max_iter_of(h);
    int done = 0, last = 0;
    rve_status st = RVE_OK;
    for (h->inc_it0 = 0; h->inc_it0 < max_iter && !done; h->inc_it0 += h->inc_nb) {
      if ((st = enqueue_iterations<T>(h))) break;
      cudaError_t e = cudaEventSynchronize(h->ev_sync);
      if (e != cudaSuccess) {
        st = cuda_fail(h, e, "adjoint iterations");
        break;
      }
      tcollect(h, h->inc_nb);
      done = h->st_host->done;
      last = h->st_host->done_it;
    }
    if (st == RVE_OK && done == 1) {
      XArgs<T> ca = x_args<T>(h, h->spec[r.s_in(last)], nullptr, last);
      cudaError_t e = launch_xpass<T>(ca, kLinearLaw, true, h->xgrid, xsmem_total(h), s);
      if (e != cudaSuccess) st = cuda_fail(h, e, "adjoint commit");
    } else if (st == RVE_OK) {
      st = fail(h, done == 2 ? RVE_ERR_NAN : RVE_ERR_NOT_CONVERGED, "adjoint fixed point did not converge");
    }
    h->lin_mode = false;
    h->lin_B = h->lin_g = nullptr;
    h->lin_mu = nullptr;
    h->lin_sref = 0.0;
    if (st) return st;
    if (iters) *iters += last + 1;
  }
  // constraint part: stress adjoint -w mu, no state adjoint
  RVE_CUDA(h, launch_adj<T>(3, n, s, at(kAdjMu), nullptr, nullptr, at(kAdjSigB), nullptr, nullptr));
  RVE_CUDA(h, cudaMemsetAsync(at(kAdjStZ), 0, 34 * N * sizeof(T), s));
  RVE_CUDA(h, launch_material_point_vjp<T>(M, np, n, at(kAdjRvox), at(kAdjEpsP), at(kAdjEpsC), at(kAdjStP), dt, nsub,
                                           at(kAdjSigB), at(kAdjStZ), at(kAdjDummy), at(kAdjEnB), at(kAdjRbB),
                                           at(kAdjPbB), tab, s));
  // outputs: state and strain adjoints at t_{n-1} (double, device)
  RVE_CUDA(h, launch_adj<T>(5, 34 * n, s, at(kAdjStB), at(kAdjStZ), nullptr, state_b, nullptr, nullptr));
  RVE_CUDA(h, launch_adj<T>(5, 6 * n, s, at(kAdjEnA), at(kAdjEnB), nullptr, eps_b, nullptr, nullptr));
  // parameter and rotation adjoints: per-voxel values summed on the device in a fixed order
  // (parameters: block partials, added here; rotations: per grain over the grain-sorted
  // voxel list), into the unused-output slot
  if (!h->adj_perm) {
    std::vector<int> goff((size_t)h->n_grains + 1, 0);
    for (size_t i = 0; i < N; ++i) ++goff[(size_t)h->gid_host[i] + 1];
    for (int g = 0; g < h->n_grains; ++g) goff[g + 1] += goff[g];
    std::vector<uint32_t> perm(N);
    std::vector<int> fill(goff.begin(), goff.end() - 1);
    for (size_t i = 0; i < N; ++i) perm[(size_t)fill[h->gid_host[i]]++] = (uint32_t)i;
    rve_status st = dalloc(h, &h->adj_perm, N * sizeof(uint32_t));
    if (st) return st;
    st = dalloc(h, &h->adj_goff, goff.size() * sizeof(int));
    if (st) return st;
    RVE_CUDA(h, cudaMemcpyAsync(h->adj_perm, perm.data(), N * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    RVE_CUDA(h, cudaMemcpyAsync(h->adj_goff, goff.data(), goff.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    RVE_CUDA(h, cudaStreamSynchronize(s));
  }
  const size_t nb = (N + 255) / 256;
  if ((nb + (size_t)h->n_grains) * 9 * sizeof(double) > (size_t)30 * N * sizeof(T))
    return fail(h, RVE_ERR_UNSUPPORTED, "adjoint: more grains than the gradient scratch holds");
  double* param_part = (double*)at(kAdjDummy);
  double* grain_out = param_part + nb * 9;
  RVE_CUDA(h, launch_adj_sums<T>(at(kAdjPbA), at(kAdjPbB), at(kAdjRbA), at(kAdjRbB), (const uint32_t*)h->adj_perm,
                                 (const int*)h->adj_goff, h->n_grains, n, param_part, grain_out, s));
  std::vector<double> hp(nb * 9), Rb((size_t)h->n_grains * 9);
  RVE_CUDA(h, cudaMemcpyAsync(hp.data(), param_part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  RVE_CUDA(h, cudaMemcpyAsync(Rb.data(), grain_out, Rb.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  RVE_CUDA(h, cudaStreamSynchronize(s));
  for (int k = 0; k < 9; ++k) {
    double acc = 0.0;
    for (size_t b = 0; b < nb; ++b) acc += hp[b * 9 + k];
    pgrad[k] += acc;
  }
  for (int g = 0; g < h->n_grains; ++g) {
    double dR[3][9];
    bunge_grad(&h->euler[3 * g], dR);
    for (int k = 0; k < 3; ++k) {
      double acc = 0.0;
      for (int i = 0; i < 9; ++i) acc += Rb[(size_t)g * 9 + i] * dR[k][i];
      egrad[3 * g + k] += acc;
    }
  }
  return RVE_OK;
}

bool valid_len(int n) {
  FftDim d;
  return n >= 1 && factor_radices(n, &d);
}

bool valid_grid(int nx, int ny, int nz) {
  return nx >= 2 && nx % 2 == 0 && valid_len(nx) && valid_len(ny) && valid_len(nz);
}

template <typename T>
rve_status get_field_t(rve_s* h, int which, int dtype, void* dst, size_t bytes, int on_dev) {
  const void* src = nullptr;
  int comps = 0;
  double scale = 1.0;
  switch (which) {
    case RVE_FIELD_STRESS: src = h->sig_n; comps = 6; break;
    case RVE_FIELD_STRAIN: src = h->eps_n; comps = 6; break;
    case RVE_FIELD_EPS_P: src = h->ep; comps = 6; break;
    case RVE_FIELD_V: src = h->v; comps = 16; break;
    case RVE_FIELD_ALPHA: src = h->al; comps = 12; break;
    case RVE_FIELD_VM: src = h->sig_n; comps = 1; break;
    case RVE_FIELD_F:  // f = sqrt(2) v of the 4 twin systems (components 12..15 of v)
      src = (const T*)h->v + 12 * (size_t)h->nvox;
      comps = 4;
      scale = 1.41421356237309504880;
      break;
    default: return fail(h, RVE_ERR_INVALID_ARG, "unknown field");
  }
  if (dtype != RVE_DTYPE_F64 && dtype != RVE_DTYPE_F32) return fail(h, RVE_ERR_INVALID_ARG, "unknown dtype");
  const size_t n = (size_t)comps * h->nvox;
  const size_t elem = dtype == RVE_DTYPE_F64 ? sizeof(double) : sizeof(float);
  if (!dst || bytes < n * elem) return fail(h, RVE_ERR_INVALID_ARG, "destination too small");
  // the field in double on the device (in dst itself when it is a device double array),
  // then narrowed and / or copied to the destination
  const bool direct = on_dev && dtype == RVE_DTYPE_F64;
  double* out = (double*)dst;
  void* tmp = nullptr;
  void* tmp32 = nullptr;
  if (!direct) {
    rve_status s = dalloc(h, &tmp, n * sizeof(double));
    if (s) return s;
    out = (double*)tmp;
  }
  if (dtype == RVE_DTYPE_F32 && !on_dev) {
    rve_status s = dalloc(h, &tmp32, n * sizeof(float));
    if (s) {
      h->owned.pop_back();
      if (h->opt.free) h->opt.free(tmp, h->opt.alloc_ctx);
      else cudaFree(tmp);
      return s;
    }
  }
  cudaError_t e = which == RVE_FIELD_VM ? launch_von_mises<T>((const T*)src, out, h->nvox, h->stream)
                                        : launch_to_double<T>((const T*)src, out, (long long)n, h->stream, scale);
  if (dtype == RVE_DTYPE_F32) {
    float* f32 = on_dev ? (float*)dst : (float*)tmp32;
    if (e == cudaSuccess) e = launch_to_float<T>(out, f32, (long long)n, h->stream);
    if (e == cudaSuccess && !on_dev) e = cudaMemcpyAsync(dst, f32, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
  } else if (e == cudaSuccess && !on_dev) {
    e = cudaMemcpyAsync(dst, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  for (void* t : {tmp32, tmp}) {  // the last allocations first, as dalloc recorded them
    if (!t) continue;
    h->owned.pop_back();
    if (h->opt.free) h->opt.free(t, h->opt.alloc_ctx);
    else cudaFree(t);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "get_fields");
  return RVE_OK;
}

struct BlobHeader {
  char magic[8];
  int nx, ny, nz, precision, increment, pad;
  double time, E_n[6], E_prev[6];
  long long n_hist;
};

}  // namespace

namespace rve {
void set_global_error(const std::string& msg) { g_err = msg; }
}  // namespace rve

// ================================================================= C ABI ==============
extern "C" {

void rve_options_default(rve_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = RVE_FP64;
  o->green = RVE_GREEN_WILLOT;
  o->n_sub = 0;
  o->max_iter = 1000;
  o->fixed_iters = 0;
  o->tol = 1e-6;
  o->graphs = 1;
  o->autotune = 1;
  o->y_tile = 0;
  o->z_tile = 0;
  o->batch_group = 0;
}

void rve_material_default(rve_material* m) {
  if (!m) return;
  m->C11 = 183000.0; m->C12 = 74000.0; m->C13 = 74000.0; m->C33 = 178000.0; m->C44 = 105000.0; m->C66 = 78000.0;
  m->r0_ord = 90.0; m->r0_sup = 200.0; m->r0_twin = 110.0;
  m->K = 10.0; m->n = 10.0; m->Kt = 10.0; m->nt = 10.0;
  m->Q_s = 20.0; m->Q_b = 20.0; m->b_s = 5.0; m->b_b = 5.0;
  m->h_diag = 1.0; m->h_off = 1.2;
  m->c = 10000.0; m->d = 500.0;
  m->Kc = 1.45; m->fm = 0.8; m->eta = 1.0e4;
}

rve_status rve_create(rve_t* out, int nx, int ny, int nz, const uint32_t* grain_id, int grain_id_on_device,
                      int n_grains, const double* euler, const rve_options* opt) {
  NvtxRange range("rve_create");
  if (!out) return fail(nullptr, RVE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!grain_id || !euler || n_grains < 1) return fail(nullptr, RVE_ERR_INVALID_ARG, "need grain_id, euler, n_grains >= 1");
  if (!valid_grid(nx, ny, nz))
    return fail(nullptr, RVE_ERR_UNSUPPORTED, "grid sizes must be 2^a 3^b 5^c, at most 512, nx even");
  rve_options o;
  rve_options_default(&o);
  if (opt) o = *opt;
  if (o.precision != RVE_FP64 && o.precision != RVE_FP32) return fail(nullptr, RVE_ERR_INVALID_ARG, "bad precision");
  if (o.y_tile < 0 || o.y_tile > 16 || o.z_tile < 0 || o.z_tile > 16)
    return fail(nullptr, RVE_ERR_INVALID_ARG, "y_tile and z_tile must be in 0..16");
  if (o.green != RVE_GREEN_WILLOT && o.green != RVE_GREEN_MS) return fail(nullptr, RVE_ERR_INVALID_ARG, "bad green");
  if (o.n_sub < 0 || o.fixed_iters < 0 || o.max_iter < 0 || !(o.tol > 0)) return fail(nullptr, RVE_ERR_INVALID_ARG, "bad options");
  if ((o.alloc == nullptr) != (o.free == nullptr)) return fail(nullptr, RVE_ERR_INVALID_ARG, "alloc and free go together");
  if ((o.c0_mu != 0.0 || o.c0_lambda != 0.0) &&
      !(std::isfinite(o.c0_mu) && std::isfinite(o.c0_lambda) && o.c0_mu > 0.0 && 3.0 * o.c0_lambda + 2.0 * o.c0_mu > 0.0))
    return fail(nullptr, RVE_ERR_INVALID_ARG, "the reference medium needs c0_mu > 0 and 3 c0_lambda + 2 c0_mu > 0");
  for (long long i = 0; i < 3LL * n_grains; ++i)
    if (!std::isfinite(euler[i])) return fail(nullptr, RVE_ERR_INVALID_ARG, "euler angle not finite");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(nullptr, RVE_ERR_CUDA, "no CUDA device available");
  }
  if (o.device < 0 || o.device >= ndev) return fail(nullptr, RVE_ERR_INVALID_ARG, "bad device ordinal");
  e = cudaSetDevice(o.device);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");

  rve_s* h = new rve_s();
  h->opt = o;
  rve_material_default(&h->mat);
  h->nx = nx; h->ny = ny; h->nz = nz;
  h->H = nx / 2 + 1;
  h->NL = (long long)ny * nz;
  h->nvox = (long long)nx * ny * nz;
  h->n_grains = n_grains;
  h->stream = o.stream ? (cudaStream_t)o.stream : cudaStreamPerThread;
  h->tsize = o.precision == RVE_FP64 ? 8 : 4;
  factor_radices(nx, &h->dx);
  factor_radices(ny, &h->dy);
  factor_radices(nz, &h->dz);
  h->euler.assign(euler, euler + 3LL * n_grains);
  set_reference_medium(h->opt, h->mat, &h->lam0, &h->mu0);
  rve_status s;
  // grain map: validate on the host copy
  std::vector<uint32_t> gid((size_t)h->nvox);
  if (grain_id_on_device) {
    e = cudaMemcpy(gid.data(), grain_id, gid.size() * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { s = cuda_fail(h, e, "grain_id copy"); rve_destroy(h); return s; }
  } else {
    std::memcpy(gid.data(), grain_id, gid.size() * 4);
  }
  for (uint32_t g : gid)
    if (g >= (uint32_t)n_grains) { s = fail(h, RVE_ERR_INVALID_ARG, "grain id >= n_grains"); rve_destroy(h); return s; }
  h->gid_host = gid;
  if ((s = dalloc(h, (void**)&h->grain, gid.size() * 4))) { rve_destroy(h); return s; }
  e = cudaMemcpyAsync(h->grain, gid.data(), gid.size() * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) { s = cuda_fail(h, e, "grain_id upload"); rve_destroy(h); return s; }
  if (o.precision == RVE_FP64) {
    if ((s = upload_tables<double>(h)) || (s = alloc_fields<double>(h)) || (s = upload_root_tab<double>(h))) {
      rve_destroy(h);
      return s;
    }
  } else {
    if ((s = upload_tables<float>(h)) || (s = alloc_fields<float>(h)) || (s = upload_root_tab<float>(h))) {
      rve_destroy(h);
      return s;
    }
  }
  e = cudaEventCreateWithFlags(&h->ev_sync, cudaEventDisableTiming);
  if (e != cudaSuccess) { s = cuda_fail(h, e, "cudaEventCreate"); rve_destroy(h); return s; }
  if (o.timing)
    for (int k = 0; k < kTSlots; ++k) {
      e = cudaEventCreate(&h->ev_a[k]);
      if (e == cudaSuccess) e = cudaEventCreate(&h->ev_b[k]);
      if (e != cudaSuccess) { s = cuda_fail(h, e, "cudaEventCreate"); rve_destroy(h); return s; }
    }
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) { s = cuda_fail(h, e, "create"); rve_destroy(h); return s; }
  *out = h;
  return RVE_OK;
}

rve_status rve_set_material(rve_t h, const rve_material* m) {
  if (!h || !m) return fail(h, RVE_ERR_INVALID_ARG, "NULL argument");
  if (h->increment > 0) return fail(h, RVE_ERR_STATE, "material is fixed once stepping started");
  rve_status s = check_material(h, *m);
  if (s) return s;
  h->mat = *m;
  set_reference_medium(h->opt, h->mat, &h->lam0, &h->mu0);
  drop_graphs(h);  // the material is baked into the increment graphs
  return h->opt.precision == RVE_FP64 ? upload_root_tab<double>(h) : upload_root_tab<float>(h);
}

rve_status rve_set_mixed_load(rve_t h, const double Edot[6], const uint8_t ctrl[6], const double Sigma[6], double dt) {
  if (!h || !Edot || !ctrl || !Sigma) return fail(h, RVE_ERR_INVALID_ARG, "NULL argument");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(h, RVE_ERR_INVALID_ARG, "dt must be > 0");
  int nc = 0;
  for (int c = 0; c < 6; ++c) {
    if (!std::isfinite(Edot[c]) || !std::isfinite(Sigma[c])) return fail(h, RVE_ERR_INVALID_ARG, "load not finite");
    nc += ctrl[c] ? 1 : 0;
  }
  if (nc == 0) return fail(h, RVE_ERR_INVALID_ARG, "at least one component must be strain-controlled");
  bool same = dt == h->dt;
  for (int c = 0; c < 6; ++c)
    same = same && Edot[c] == h->Edot[c] && (ctrl[c] ? 1 : 0) == h->ctrl[c] && Sigma[c] == h->Sigma[c];
  if (same) return RVE_OK;  // unchanged load: the increment graphs stay valid
  for (int c = 0; c < 6; ++c) {
    h->Edot[c] = Edot[c];
    h->ctrl[c] = ctrl[c] ? 1 : 0;
    h->Sigma[c] = Sigma[c];
  }
  h->dt = dt;
  drop_graphs(h);  // the load and dt are baked into the increment graphs
  return RVE_OK;
}

rve_status rve_step(rve_t h, int n, long long* iters) {
  if (!h) return fail(h, RVE_ERR_INVALID_ARG, "NULL handle");
  if (n < 0) return fail(h, RVE_ERR_INVALID_ARG, "n_increments < 0");
  if (iters) *iters = 0;
  cudaError_t e = cudaSetDevice(h->opt.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  for (int i = 0; i < n; ++i) {
    rve_status s = step_one(h, iters);
    if (s) return s;
  }
  return RVE_OK;
}

rve_status rve_step_batch(rve_t* hs, int n, int n_increments, long long* iters, int* failed) {
  NvtxRange range("rve_step_batch");
  if (failed) *failed = -1;
  if (iters) *iters = 0;
  if (n < 0 || n_increments < 0 || (n > 0 && !hs)) return fail(nullptr, RVE_ERR_INVALID_ARG, "bad batch arguments");
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return fail(nullptr, RVE_ERR_INVALID_ARG, "NULL handle in the batch");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(nullptr, RVE_ERR_INVALID_ARG, "a handle is listed twice in the batch");
    if (hs[i]->opt.device != hs[0]->opt.device)
      return fail(nullptr, RVE_ERR_INVALID_ARG, "all handles of a batch must be on one device");
  }
  if (n == 0 || n_increments == 0) return RVE_OK;
  cudaError_t e = cudaSetDevice(hs[0]->opt.device);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
  if (groupable(hs, n))
    return hs[0]->opt.precision == RVE_FP64 ? step_batch_group<double>(hs, n, n_increments, iters, failed)
                                            : step_batch_group<float>(hs, n, n_increments, iters, failed);
  // Each handle runs on a private stream, ordered after the work already enqueued on its
  // own stream and before anything enqueued there after this call.
  std::vector<cudaStream_t> orig(n), priv(n, nullptr);
  rve_status first = RVE_OK;
  int first_i = -1;
  auto note = [&](int i, rve_status st) {
    if (st != RVE_OK && first == RVE_OK) {
      first = st;
      first_i = i;
    }
  };
  int made = 0;
  for (; made < n; ++made) {
    rve_s* h = hs[made];
    orig[made] = h->stream;
    e = cudaStreamCreateWithFlags(&priv[made], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_sync, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(priv[made], h->ev_sync, 0);
    if (e != cudaSuccess) {
      note(made, cuda_fail(h, e, "batch stream set-up"));
      if (priv[made]) cudaStreamDestroy(priv[made]);
      break;
    }
    h->stream = priv[made];
  }
  std::vector<int> left(n, n_increments);
  std::vector<char> active(n, 0);
  int n_active = 0;
  if (first == RVE_OK)
    for (int i = 0; i < n; ++i) {
      rve_status st = inc_begin_any(hs[i]);
      if (st) note(i, st);
      else { active[i] = 1; ++n_active; }
    }
  // Round-robin over the handles: resume each one whose last enqueued phase finished.
  while (n_active > 0) {
    bool progressed = false;
    for (int i = 0; i < n; ++i) {
      if (!active[i]) continue;
      rve_s* h = hs[i];
      const cudaError_t q = cudaEventQuery(h->ev_sync);
      if (q == cudaErrorNotReady) continue;
      progressed = true;
      bool fin = false;
      rve_status st;
      if (q != cudaSuccess) {
        h->inc_phase = 0;
        st = cuda_fail(h, q, "cudaEventQuery");
      } else {
        st = inc_advance_any(h, &fin, iters);
      }
      if (st == RVE_OK && fin && --left[i] > 0) st = inc_begin_any(h);
      if (st != RVE_OK || (fin && left[i] == 0)) {
        note(i, st);
        active[i] = 0;
        --n_active;
      }
    }
    if (!progressed) std::this_thread::yield();
  }
  for (int i = 0; i < made; ++i) {
    rve_s* h = hs[i];
    e = cudaEventRecord(h->ev_sync, priv[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(orig[i], h->ev_sync, 0);
    if (e != cudaSuccess) note(i, cuda_fail(h, e, "batch stream join"));
    h->stream = orig[i];
    cudaStreamDestroy(priv[i]);
  }
  if (failed) *failed = first_i;
  if (first != RVE_OK) g_err = "handle " + std::to_string(first_i) + ": " + hs[first_i]->err;
  return first;
}

rve_status rve_batch_grouped(rve_t* hs, int n, int* grouped) {
  if (!grouped || n < 0 || (n > 0 && !hs)) return fail(nullptr, RVE_ERR_INVALID_ARG, "bad batch arguments");
  for (int i = 0; i < n; ++i)
    if (!hs[i]) return fail(nullptr, RVE_ERR_INVALID_ARG, "NULL handle in the batch");
  *grouped = groupable(hs, n) ? 1 : 0;
  return RVE_OK;
}

rve_status rve_adjoint_increment(rve_t h, const double* eps_prev, const double* eps_cur, const double* state_prev,
                                 const double dS[6], double dt, double* state_b, double* eps_b, double* param_grad,
                                 double* euler_grad, long long* iterations_out) {
  NvtxRange range("rve_adjoint_increment");
  if (!h) return fail(h, RVE_ERR_INVALID_ARG, "NULL handle");
  if (!eps_prev || !eps_cur || !state_prev || !dS || !state_b || !eps_b || !param_grad || !euler_grad ||
      !(dt > 0))
    return fail(h, RVE_ERR_INVALID_ARG, "bad adjoint arguments");
  cudaError_t e = cudaSetDevice(h->opt.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  drop_graphs(h);  // the adjoint solve reuses the spectra; the forward state is not kept
  return h->opt.precision == RVE_FP64
             ? adjoint_increment<double>(h, eps_prev, eps_cur, state_prev, dS, dt, state_b, eps_b, param_grad,
                                         euler_grad, iterations_out)
             : adjoint_increment<float>(h, eps_prev, eps_cur, state_prev, dS, dt, state_b, eps_b, param_grad,
                                        euler_grad, iterations_out);
}

rve_status rve_get_effective(rve_t h, rve_effective* last, rve_effective* hist, int cap, int* n_hist) {
  if (!h) return fail(h, RVE_ERR_INVALID_ARG, "NULL handle");
  if (n_hist) *n_hist = (int)h->hist.size();
  if (last) {
    if (h->hist.empty()) std::memset(last, 0, sizeof(*last));
    else *last = h->hist.back();
  }
  if (hist && cap > 0) {
    const int m = std::min<int>(cap, (int)h->hist.size());
    for (int i = 0; i < m; ++i) hist[i] = h->hist[i];
  }
  return RVE_OK;
}

rve_status rve_get_fields_as(rve_t h, int which, int dtype, void* dst, size_t bytes, int on_dev) {
  if (!h) return fail(h, RVE_ERR_INVALID_ARG, "NULL handle");
  cudaError_t e = cudaSetDevice(h->opt.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  return h->opt.precision == RVE_FP64 ? get_field_t<double>(h, which, dtype, dst, bytes, on_dev)
                                      : get_field_t<float>(h, which, dtype, dst, bytes, on_dev);
}

rve_status rve_get_fields(rve_t h, int which, void* dst, size_t bytes, int on_dev) {
  return rve_get_fields_as(h, which, RVE_DTYPE_F64, dst, bytes, on_dev);
}

rve_status rve_save_state(rve_t h, void* blob, size_t* bytes) {
  if (!h || !bytes) return fail(h, RVE_ERR_INVALID_ARG, "NULL argument");
  const size_t ts = h->tsize;
  const size_t spec = (size_t)6 * h->NL * h->H * 2 * ts;
  const size_t fld = (size_t)h->nvox * ts;
  const size_t need = sizeof(BlobHeader) + h->hist.size() * sizeof(rve_effective) + 2 * spec + fld * (6 + 16 + 12 + 6 + 6);
  if (!blob) {
    *bytes = need;
    return RVE_OK;
  }
  if (*bytes < need) return fail(h, RVE_ERR_INVALID_ARG, "blob too small");
  BlobHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "RVESTAT1", 8);
  hd.nx = h->nx; hd.ny = h->ny; hd.nz = h->nz; hd.precision = h->opt.precision; hd.increment = h->increment;
  hd.time = h->time;
  std::memcpy(hd.E_n, h->E_n, sizeof(hd.E_n));
  std::memcpy(hd.E_prev, h->E_prev, sizeof(hd.E_prev));
  hd.n_hist = (long long)h->hist.size();
  char* p = (char*)blob;
  std::memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  if (!h->hist.empty()) std::memcpy(p, h->hist.data(), h->hist.size() * sizeof(rve_effective));
  p += h->hist.size() * sizeof(rve_effective);
  struct { const void* d; size_t n; } parts[] = {{h->spec[h->sb], spec}, {h->P[h->pb], spec}, {h->ep, 6 * fld},
                                                 {h->v, 16 * fld},     {h->al, 12 * fld},   {h->eps_n, 6 * fld},
                                                 {h->sig_n, 6 * fld}};
  for (auto& q : parts) {
    cudaError_t e = cudaMemcpyAsync(p, q.d, q.n, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "save_state");
    p += q.n;
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "save_state");
  *bytes = need;
  return RVE_OK;
}

rve_status rve_load_state(rve_t h, const void* blob, size_t bytes) {
  if (!h || !blob) return fail(h, RVE_ERR_INVALID_ARG, "NULL argument");
  if (bytes < sizeof(BlobHeader)) return fail(h, RVE_ERR_INVALID_ARG, "blob too small");
  BlobHeader hd;
  std::memcpy(&hd, blob, sizeof(hd));
  if (std::memcmp(hd.magic, "RVESTAT1", 8) || hd.nx != h->nx || hd.ny != h->ny || hd.nz != h->nz ||
      hd.precision != h->opt.precision || hd.n_hist < 0)
    return fail(h, RVE_ERR_INVALID_ARG, "blob does not match this handle");
  const size_t ts = h->tsize;
  const size_t spec = (size_t)6 * h->NL * h->H * 2 * ts;
  const size_t fld = (size_t)h->nvox * ts;
  const size_t need = sizeof(BlobHeader) + (size_t)hd.n_hist * sizeof(rve_effective) + 2 * spec + fld * 46;
  if (bytes < need) return fail(h, RVE_ERR_INVALID_ARG, "blob truncated");
  const char* p = (const char*)blob + sizeof(hd);
  h->hist.assign((const rve_effective*)p, (const rve_effective*)p + hd.n_hist);
  p += (size_t)hd.n_hist * sizeof(rve_effective);
  struct { void* d; size_t n; } parts[] = {{h->spec[h->sb], spec}, {h->P[h->pb], spec}, {h->ep, 6 * fld},
                                           {h->v, 16 * fld},     {h->al, 12 * fld},   {h->eps_n, 6 * fld},
                                           {h->sig_n, 6 * fld}};
  for (auto& q : parts) {
    cudaError_t e = cudaMemcpyAsync(q.d, p, q.n, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "load_state");
    p += q.n;
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "load_state");
  h->increment = hd.increment;
  h->time = hd.time;
  std::memcpy(h->E_n, hd.E_n, sizeof(hd.E_n));
  std::memcpy(h->E_prev, hd.E_prev, sizeof(hd.E_prev));
  return RVE_OK;
}

rve_status rve_kernel_times(rve_t h, double* ms, long long* launches, int reset) {
  if (!h) return fail(h, RVE_ERR_INVALID_ARG, "NULL handle");
  if (!h->opt.timing) return fail(h, RVE_ERR_STATE, "handle created without timing");
  for (int k = 0; k < RVE_K_COUNT; ++k) {
    if (ms) ms[k] = h->k_ms[k];
    if (launches) launches[k] = h->k_n[k];
    if (reset) {
      h->k_ms[k] = 0.0;
      h->k_n[k] = 0;
    }
  }
  return RVE_OK;
}

rve_status rve_get_residuals(rve_t h, double* e_eq, double* c_F, int cap, int* n) {
  if (!h) return fail(h, RVE_ERR_INVALID_ARG, "NULL handle");
  const int m = (int)h->res_e.size();
  if (n) *n = m;
  for (int i = 0; i < std::min(cap, m); ++i) {
    if (e_eq) e_eq[i] = h->res_e[i];
    if (c_F) c_F[i] = h->res_c[i];
  }
  return RVE_OK;
}

const char* rve_last_error(rve_t h) {
  if (h) return h->err.c_str();
  return g_err.c_str();
}

void rve_destroy(rve_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  release(h);
  delete h;
}

rve_status rve_material_point(int precision, const rve_material* mat, long long nvox, const void* R, const void* eps_n,
                              const void* eps, void* state, void* sigma, double dt, int n_sub, void* stream) {
  if (!mat || nvox < 0 || (nvox > 0 && (!R || !eps_n || !eps || !state || !sigma)) || !(dt > 0) || n_sub < 1)
    return fail(nullptr, RVE_ERR_INVALID_ARG, "bad material-point arguments");
  rve_s tmp;
  tmp.mat = *mat;
  rve_status s = check_material(&tmp, *mat);
  if (s) return fail(nullptr, s, tmp.err);
  reference_medium(tmp.mat, &tmp.lam0, &tmp.mu0);
  if (precision != RVE_FP64 && precision != RVE_FP32) return fail(nullptr, RVE_ERR_INVALID_ARG, "bad precision");
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  tmp.stream = st;
  const int np = rate_variant(mat->eta, mat->K, mat->Kt, is_small_int(mat->n), is_small_int(mat->nt));
  s = precision == RVE_FP64 ? upload_root_tab<double>(&tmp) : upload_root_tab<float>(&tmp);
  if (s) {
    release(&tmp);
    return fail(nullptr, s, tmp.err);
  }
  cudaError_t e;
  if (precision == RVE_FP64)
    e = launch_material_point<double>(make_mat<double>(&tmp), np, nvox, (const double*)R, (const double*)eps_n,
                                      (const double*)eps, (double*)state, (double*)sigma, dt, n_sub,
                                      (const double*)tmp.root_tab, st);
  else
    e = launch_material_point<float>(make_mat<float>(&tmp), np, nvox, (const float*)R, (const float*)eps_n,
                                     (const float*)eps, (float*)state, (float*)sigma, (float)dt, n_sub,
                                     (const float*)tmp.root_tab, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  release(&tmp);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "material_point");
  return RVE_OK;
}

rve_status rve_material_point_vjp(int precision, const rve_material* mat, long long nvox, const void* R,
                                  const void* eps_n, const void* eps, const void* state, const void* sigma_b,
                                  void* state_b, void* eps_b, void* eps_n_b, void* R_b, void* param_b, double dt,
                                  int n_sub, void* stream) {
  if (!mat || nvox < 0 || (nvox > 0 && (!R || !eps_n || !eps || !state || !sigma_b || !state_b || !eps_b ||
                                        !eps_n_b || !R_b || !param_b)) ||
      !(dt > 0) || n_sub < 1 || n_sub > kMaxSubVjp)
    return fail(nullptr, RVE_ERR_INVALID_ARG, "bad material-point adjoint arguments (n_sub must be 1..16)");
  rve_s tmp;
  tmp.mat = *mat;
  rve_status s = check_material(&tmp, *mat);
  if (s) return fail(nullptr, s, tmp.err);
  reference_medium(tmp.mat, &tmp.lam0, &tmp.mu0);
  if (precision != RVE_FP64 && precision != RVE_FP32) return fail(nullptr, RVE_ERR_INVALID_ARG, "bad precision");
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  tmp.stream = st;
  const int np = rate_variant(mat->eta, mat->K, mat->Kt, is_small_int(mat->n), is_small_int(mat->nt));
  s = precision == RVE_FP64 ? upload_root_tab<double>(&tmp) : upload_root_tab<float>(&tmp);
  if (s) {
    release(&tmp);
    return fail(nullptr, s, tmp.err);
  }
  cudaError_t e;
  if (precision == RVE_FP64)
    e = launch_material_point_vjp<double>(make_mat<double>(&tmp), np, nvox, (const double*)R, (const double*)eps_n,
                                          (const double*)eps, (const double*)state, dt, n_sub,
                                          (const double*)sigma_b, (double*)state_b, (double*)eps_b,
                                          (double*)eps_n_b, (double*)R_b, (double*)param_b,
                                          (const double*)tmp.root_tab, st);
  else
    e = launch_material_point_vjp<float>(make_mat<float>(&tmp), np, nvox, (const float*)R, (const float*)eps_n,
                                         (const float*)eps, (const float*)state, (float)dt, n_sub,
                                         (const float*)sigma_b, (float*)state_b, (float*)eps_b, (float*)eps_n_b,
                                         (float*)R_b, (float*)param_b, (const float*)tmp.root_tab, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  release(&tmp);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "material_point_vjp");
  return RVE_OK;
}

}  // extern "C"

// Twiddle tables of the stand-alone transforms, cached per (device, precision, length) like
// an FFT plan: built on first use (cudaMalloc and a synchronous copy), never modified
// afterwards, kept until the process exits (2 n values each).
struct TwiddleEntry {
  int dev, elem, n;
  void* ptr;
};
std::mutex g_twiddle_mu;
std::vector<TwiddleEntry> g_twiddles;

template <typename T>
static cudaError_t cached_twiddles(int n, const C2<T>** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_twiddle_mu);
  for (const TwiddleEntry& t : g_twiddles)
    if (t.dev == dev && t.elem == (int)sizeof(T) && t.n == n) {
      *out = (const C2<T>*)t.ptr;
      return cudaSuccess;
    }
  std::vector<T> host(2 * (size_t)n);
  fill_twiddles<T>(n, host.data());
  void* p = nullptr;
  if ((e = cudaMalloc(&p, host.size() * sizeof(T))) != cudaSuccess) return e;
  if ((e = cudaMemcpy(p, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaFree(p);
    return e;
  }
  g_twiddles.push_back(TwiddleEntry{dev, (int)sizeof(T), n, p});
  *out = (const C2<T>*)p;
  return cudaSuccess;
}

template <typename T>
static rve_status fft_t(int nx, int ny, int nz, int ncomp, const void* in, void* spec, void* out, int sign,
                        cudaStream_t st) {
  FftDim dx, dy, dz;
  factor_radices(nx, &dx);
  factor_radices(ny, &dy);
  factor_radices(nz, &dz);
  const int H = nx / 2 + 1;
  const long long NL = (long long)ny * nz;
  const C2<T> *tw_x = nullptr, *tw_y = nullptr, *tw_z = nullptr;
  cudaError_t e = cached_twiddles<T>(nx, &tw_x);
  if (e == cudaSuccess) e = cached_twiddles<T>(ny, &tw_y);
  if (e == cudaSuccess) e = cached_twiddles<T>(nz, &tw_z);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "fft twiddle tables");
  // x: up to 32 lines (16 packed pairs) of one component per CTA
  const int L = std::max(1, std::min(32, 4096 / nx));
  XFftArgs<T> xa{};
  xa.nx = nx; xa.H = H; xa.L = L; xa.ncomp = ncomp; xa.NL = NL;
  xa.dx = dx;
  xa.tw = tw_x;
  xa.real = (const T*)in;
  xa.spec = (C2<T>*)spec;
  xa.real_out = (T*)out;
  const size_t xsm = (size_t)(nx + 2 * ((L + 1) / 2) * (nx + 1)) * sizeof(C2<T>);
  const dim3 xg((unsigned)((NL + L - 1) / L), ncomp);
  const size_t budget = 96 * 1024;
  // y and z: one component's kx chunk per CTA; lengths with a register split take the
  // two-step kernel with the chunks of H split evenly (at most 384 / N1 columns each), the
  // others Stockham passes on a chunk sized for the shared-memory budget
  auto pass = [&](const FftDim& d, const C2<T>* tw, long long stride, int n_o2, long long A, long long B,
                  int n_outer) {
    LineArgs<T> la{};
    la.done = nullptr;  // stand-alone transform: always runs
    la.d = d;
    la.tw = tw;
    la.spec = (C2<T>*)spec;
    la.H = H;
    const int n1 = pencil_n1(d.n);
    if (n1 > 0) {
      const int cmax = 384 / n1;
      const int chunks = (H + cmax - 1) / cmax;
      la.HC = (H + chunks - 1) / chunks;
    } else {
      la.HC = (int)std::max<size_t>(1, std::min<size_t>(16, (budget / (4 * sizeof(T))) / d.n));
      la.HC = std::min(la.HC, H);
    }
    la.n_o2 = n_o2;
    la.NC = 1;
    la.hstride = 1;
    la.stride = stride;
    la.A = A;
    la.B = B;
    const size_t sm = (size_t)(d.n + 2 * la.HC * (d.n + 1)) * 2 * sizeof(T);
    return launch_line<T>(la, sign, dim3((H + la.HC - 1) / la.HC, n_outer), sm, st);
  };
  const long long plane = (long long)nz * ny * H;
  if (e == cudaSuccess) {
    if (sign < 0) {
      e = launch_xfft<T>(xa, -1, xg, xsm, st);
      if (e == cudaSuccess) e = pass(dy, tw_y, H, nz, plane, (long long)ny * H, ncomp * nz);
      if (e == cudaSuccess) e = pass(dz, tw_z, (long long)ny * H, ny, plane, H, ncomp * ny);
    } else {
      e = pass(dz, tw_z, (long long)ny * H, ny, plane, H, ncomp * ny);
      if (e == cudaSuccess) e = pass(dy, tw_y, H, nz, plane, (long long)ny * H, ncomp * nz);
      if (e == cudaSuccess) e = launch_xfft<T>(xa, +1, xg, xsm, st);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "fft");
  return RVE_OK;
}

extern "C" {

rve_status rve_fft_r2c(int precision, int nx, int ny, int nz, int ncomp, const void* in, void* out, void* stream) {
  if (!valid_grid(nx, ny, nz)) return fail(nullptr, RVE_ERR_UNSUPPORTED, "bad size");
  if (ncomp < 1 || !in || !out) return fail(nullptr, RVE_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  if (precision == RVE_FP64) return fft_t<double>(nx, ny, nz, ncomp, in, out, nullptr, -1, st);
  if (precision == RVE_FP32) return fft_t<float>(nx, ny, nz, ncomp, in, out, nullptr, -1, st);
  return fail(nullptr, RVE_ERR_INVALID_ARG, "bad precision");
}

rve_status rve_fft_c2r(int precision, int nx, int ny, int nz, int ncomp, void* in, void* out, void* stream) {
  if (!valid_grid(nx, ny, nz)) return fail(nullptr, RVE_ERR_UNSUPPORTED, "bad size");
  if (ncomp < 1 || !in || !out) return fail(nullptr, RVE_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  if (precision == RVE_FP64) return fft_t<double>(nx, ny, nz, ncomp, nullptr, in, out, +1, st);
  if (precision == RVE_FP32) return fft_t<float>(nx, ny, nz, ncomp, nullptr, in, out, +1, st);
  return fail(nullptr, RVE_ERR_INVALID_ARG, "bad precision");
}

}  // extern "C"
