/*
 * rve.h -- C ABI of the GB300 full-field solver for polycrystalline RVEs.
 *
 * The library solves, on one GPU, the periodic voxel problem of arXiv 2402.09996:
 * small-strain Meric-Cailletaud crystal plasticity (Sec. 3) with 12 slip and 4
 * twinning pseudo-slip systems (Table 1), regularised by viscous hardening
 * (Sec. 4, Eq. (regu)), integrated explicitly per voxel with RK4 substeps and
 * coupled to a Green-operator ("FFT") fixed-point solver (Sec. 3, last paragraph),
 * under a mixed macroscopic load (Sec. 5: prescribed uniaxial strain, free stresses).
 *
 * Conventions for every call:
 *  - Symmetric tensors are 6-vectors in the order (11, 22, 33, 23, 13, 12) with
 *    tensor (not engineering) shear components.  Units: MPa and s.
 *  - Voxel (i, j, k) of an nx*ny*nz grid has flat index i + nx*(j + ny*k), x fastest;
 *    its centre is ((i+1/2)/nx, (j+1/2)/ny, (k+1/2)/nz) in the unit periodic cell.
 *  - Host input arrays are copied during the call; the caller keeps ownership and
 *    may free them afterwards.  Device pointers must stay valid during the call.
 *  - The handle owns its device buffers (through the optional allocator callbacks
 *    when given).  All device work is enqueued on the handle's stream; calls that
 *    return host data synchronise that stream only.
 *  - Every call returns an rve_status; RVE_OK is 0.  On failure rve_last_error()
 *    describes the cause.  After RVE_ERR_NOT_CONVERGED or RVE_ERR_NAN the handle
 *    keeps the state of the last committed increment and stays usable.
 *  - A handle is not thread-safe; distinct handles are independent.
 *  - Nothing here falls back to the CPU: without a usable CUDA device every
 *    call that needs one returns RVE_ERR_CUDA.
 */
#ifndef RVE_H
#define RVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rve_s* rve_t; /* opaque, owned by the library */

typedef enum {
  RVE_OK = 0,
  RVE_ERR_INVALID_ARG = 1,   /* bad size, pointer, option or material value */
  RVE_ERR_CUDA = 2,          /* a CUDA runtime call failed or no device */
  RVE_ERR_OOM = 3,           /* device allocation failed */
  RVE_ERR_NOT_CONVERGED = 4, /* fixed point hit max_iter; increment not committed */
  RVE_ERR_NAN = 5,           /* NaN/Inf in the averages; increment not committed */
  RVE_ERR_STATE = 6,         /* call not valid in the handle's state */
  RVE_ERR_UNSUPPORTED = 7    /* grid size or option the library does not handle */
} rve_status;

typedef enum {
  RVE_FP64 = 0, /* fields, constitutive update and reductions in double */
  RVE_FP32 = 1  /* fields and constitutive update in float; averages, norms and the
                   mixed-load update in double */
} rve_precision;

typedef enum {
  RVE_GREEN_WILLOT = 0, /* rotated scheme: kappa_j = sin(q_j/2) prod_{m!=j} cos(q_m/2) */
  RVE_GREEN_MS = 1      /* continuous frequencies, Nyquist component set to zero */
} rve_green;

typedef void* (*rve_alloc_fn)(size_t bytes, void* ctx);
typedef void (*rve_free_fn)(void* ptr, void* ctx);

typedef struct {
  int precision;      /* rve_precision */
  int green;          /* rve_green */
  int n_sub;          /* RK4 substeps per increment; 0 = smallest power of two with
                         dt / n_sub <= 1/8 s */
  int max_iter;       /* fixed-point iteration cap per increment (default 1000) */
  int fixed_iters;    /* > 0: run exactly this many iterations per increment and
                         commit the last one (parity mode); 0 = stop on tol */
  double tol;         /* equilibrium and stress-constraint tolerance (default 1e-6) */
  void* stream;       /* cudaStream_t; NULL = the per-thread default stream */
  int device;         /* CUDA device ordinal (default 0) */
  rve_alloc_fn alloc; /* optional device allocator; NULL = cudaMalloc */
  rve_free_fn free;   /* must be given together with alloc */
  void* alloc_ctx;    /* passed back to alloc/free */
  int timing;         /* nonzero: record CUDA events around every kernel launch on the
                         handle's stream and accumulate per-kernel times (rve_kernel_times) */
  int graphs;         /* nonzero (default): run each increment's fixed-point loop on the device
                         as one CUDA graph launch (a conditional while-node repeats the
                         iteration until the residual kernel decides; the commit follows in the
                         same graph), so the host waits once per increment.  The graphs are
                         built on first use per buffer rotation (three per handle) and rebuilt
                         after rve_set_mixed_load changes the load.  Ignored when timing is set. */
  int autotune;       /* nonzero (default): before the first increment, time the y and z FFT
                         passes for kx tile widths 1, 2, 4, 8, 16 on scratch buffers and keep the
                         fastest (results do not depend on the widths) */
  int y_tile, z_tile; /* > 0: force the kx tile width of the y (z) pass, overriding the
                         autotuner and the default (at most 16; clamped to nx/2 + 1) */
  int batch_group;    /* nonzero: rve_step_batch may step this handle in a group (one
                         launch per pass over all members); 0 (default) keeps it on its own
                         stream.  See rve_step_batch. */
  double c0_lambda, c0_mu; /* isotropic reference medium of the Green operator [MPa].  c0_mu > 0
                         (with 3 c0_lambda + 2 c0_mu > 0) sets it; 0, 0 (default) takes
                         3 k0 = 2 mu0 = (smallest + largest Mandel eigenvalue of C) / 2.  The
                         converged solution does not depend on it; the convergence rate does
                         (too soft a medium does not converge). */
} rve_options;

/* Kernel kinds reported by rve_kernel_times. */
typedef enum {
  RVE_K_XPASS = 0,  /* inverse x-FFT, constitutive update, polarisation, forward x-FFT */
  RVE_K_YFWD = 1,   /* forward y-FFT */
  RVE_K_ZGREEN = 2, /* forward z-FFT, Green operator, residual, inverse z-FFT */
  RVE_K_YINV = 3,   /* inverse y-FFT */
  RVE_K_COMMIT = 4, /* commit of the converged increment */
  RVE_K_SHIFT = 5,  /* uniform strain shift at the start of an increment */
  RVE_K_IDLE = 6,   /* speculative iteration launches that returned at once because the
                       increment had already converged (counted, time not accumulated) */
  RVE_K_COUNT = 7
} rve_kernel_kind;

/* Constants of Sec. 3 and Sec. 4 (MPa, s).  rve_material_default() fills the
 * tetragonal gamma-TiAl moduli (C33 = 178 GPa), r0 = 90/200/110 MPa (ordinary,
 * super, twin), K = Kt = 10, n = nt = 10, Q = 20, b = 5, interaction 1 / 1.2,
 * kinematic c = 1e4, d = 500, Kc = 1.45, fm = 0.8, eta = 1e4 MPa s. */
typedef struct {
  double C11, C12, C13, C33, C44, C66;
  double r0_ord, r0_sup, r0_twin;
  double K, n, Kt, nt;
  double Q_s, Q_b, b_s, b_b;
  double h_diag, h_off;
  double c, d;
  double Kc, fm, eta;
} rve_material;

/* One committed increment (Sec. 5 measures). */
typedef struct {
  int increment;          /* 1-based index of the committed increment */
  int iterations;         /* fixed-point iterations it took */
  double time;            /* t_{n+1} [s] */
  double E[6];            /* macroscopic strain */
  double S[6];            /* mean stress <sigma> */
  double S_eq_of_mean;    /* von Mises of <sigma> */
  double mean_S_eq;       /* <sigma_eq>, mean of the local von Mises stress */
  double mean_f;          /* <f_beta>: mean over the 4 twin systems and voxels */
  double mean_v;          /* <v^s>: mean over the 12 slip systems and voxels */
  double residual;        /* equilibrium error of the committed iterate */
  double stress_residual; /* relative error of the free mean-stress components */
} rve_effective;

typedef enum {
  RVE_FIELD_STRESS = 0, /* sigma, sample frame, 6 x nvox */
  RVE_FIELD_STRAIN = 1, /* eps, sample frame, 6 x nvox */
  RVE_FIELD_EPS_P = 2,  /* plastic strain, crystal frame, 6 x nvox */
  RVE_FIELD_V = 3,      /* accumulated slip v (12 slip + 4 twin), 16 x nvox */
  RVE_FIELD_ALPHA = 4,  /* kinematic variables of the slip systems, 12 x nvox */
  RVE_FIELD_VM = 5,     /* local von Mises stress, 1 x nvox */
  RVE_FIELD_F = 6       /* twin volume fractions f = sqrt(2) v of the 4 twin systems (Sec. 3),
                           4 x nvox */
} rve_field;

/* Element type of a field copy (rve_get_fields_as). */
typedef enum {
  RVE_DTYPE_F64 = 0, /* double */
  RVE_DTYPE_F32 = 1  /* float (exact for the fields of an RVE_FP32 handle, rounded otherwise) */
} rve_dtype;

void rve_options_default(rve_options* opt);
void rve_material_default(rve_material* mat);

/* Create a solver for an nx*ny*nz periodic RVE (Sec. 2: voxel grain map with one
 * orientation per grain).
 *   grain_id  nvox labels < n_grains (host, or device if grain_id_on_device);
 *   euler     n_grains*3 Bunge angles (phi1, Phi, phi2) in rad, host;
 *             R = Rz(phi1) Rx(Phi) Rz(phi2) maps crystal to sample axes.
 * Each of nx, ny, nz must be 2^a 3^b 5^c with n <= 512; nx even and >= 2 (ny = 1 and/or
 * nz = 1 give 2-D and 1-D periodic cells).
 * The material starts at rve_material_default(), the load at uniaxial strain rate
 * 1e-3/s along z with the other mean stresses held at zero and dt = 1 s. */
rve_status rve_create(rve_t* out, int nx, int ny, int nz, const uint32_t* grain_id,
                      int grain_id_on_device, int n_grains, const double* euler,
                      const rve_options* opt);

/* Replace the material constants (Sec. 3 elastic moduli and plasticity parameters,
 * Sec. 4 eta).  Allowed before the first step only (RVE_ERR_STATE otherwise). */
rve_status rve_set_material(rve_t h, const rve_material* mat);

/* Mixed macroscopic load for the following increments (Sec. 5 loading):
 *   Edot[6]        strain rate of the strain-controlled components [1/s];
 *   strain_ctrl[6] 1 = strain-controlled, 0 = stress-controlled;
 *   Sigma[6]       target mean stress of the stress-controlled components [MPa];
 *   dt             increment length [s], > 0.
 * At least one component must be strain-controlled. */
rve_status rve_set_mixed_load(rve_t h, const double Edot[6], const uint8_t strain_ctrl[6],
                              const double Sigma[6], double dt);

/* Run n_increments load increments; each runs the fixed point to convergence
 * (or fixed_iters) and commits.  iterations_out (host, may be NULL) receives the
 * total fixed-point iterations run by this call, committed increments only. */
rve_status rve_step(rve_t h, int n_increments, long long* iterations_out);

/* Run n_increments load increments on each of n independent solvers at once (an
 * ensemble of RVE realizations of any sizes; Sec. 5 averages over such realizations).
 * Results are identical to calling rve_step on each handle in turn.
 *  - Grouped (2 to 16 handles of one precision with the same material, load and
 *    substeps, all with graphs and batch_group on and timing off; batch_group is off by
 *    default because the private-stream mode measured faster on the ensemble
 *    workload): the handles are
 *    stepped as one group on a private stream.  Every pass of a fixed-point iteration
 *    is one kernel launch whose grid spans all members' grids (each CTA runs its
 *    member's pass unchanged), the members iterate in lockstep (a member whose
 *    increment is decided returns at once from later launches), and one increment of
 *    the whole group is one CUDA graph launch.
 *  - Otherwise each handle works on a private stream created for the call, and the host
 *    resumes each handle as soon as its enqueued iterations finish, so the RVEs' kernels
 *    run concurrently.
 * In both modes the private streams are ordered after the work already enqueued on each
 * handle's own stream and before any work enqueued there afterwards.
 *   hs             n distinct handles on one device (host array, not retained);
 *   iterations_out total committed fixed-point iterations over all handles (may be NULL);
 *   failed_out     index of the first handle that returned an error, or -1 (may be NULL).
 * A handle that fails (RVE_ERR_NOT_CONVERGED, RVE_ERR_NAN, ...) keeps its last committed
 * increment and stops; the others run all n_increments.  The first error is returned and
 * rve_last_error(NULL) names its handle.  With opt.timing the kernel times of a handle
 * include the time its kernels shared the GPU with the other handles'. */
rve_status rve_step_batch(rve_t* hs, int n, int n_increments, long long* iterations_out, int* failed_out);

/* Whether rve_step_batch would step these n handles as one group (*grouped = 1) or on
 * private streams (*grouped = 0), by the rule stated there.  No device work. */
rve_status rve_batch_grouped(rve_t* hs, int n, int* grouped);

/* Adjoint of one converged load increment n (t_{n-1} -> t_n) of a history objective J
 * (the paper defines no adjoint; this extends its method to gradients).  The objective
 * itself is the caller's: it supplies dJ/d<sigma>_n for the increment (dS) and the
 * adjoints handed back by the later increments; the Python binding's history_gradient
 * forms J = sum_n w_n (<sigma_zz>_n - target_n)^2 and its dS this way.  The increment's
 * converged strain solves the Green-operator fixed point (Sec. 4) with the mixed load; the
 * adjoint solves the transposed linearised problem (the same fixed point with the
 * transposed algorithmic tangent and the derivative of J as a source) and runs the
 * reverse pass of the constitutive update (rve_material_point_vjp) on every voxel.
 *   eps_prev, eps_cur  6*nvox committed strain at t_{n-1} and t_n (device, double);
 *   state_prev         34*nvox state at t_{n-1} (device, double; rve_get_fields layout:
 *                      eps_p 6, v 16, alpha 12, component-major);
 *   dS[6]              dJ / d<sigma>_n (host);
 *   dt                 the increment's length;
 *   state_b   34*nvox  in: dJ/d(state at t_n); out: dJ/d(state at t_{n-1}) (device, double);
 *   eps_b     6*nvox   in: dJ/d(strain at t_n) through later increments; out: the same at
 *                      t_{n-1} (device, double);
 *   param_grad[9]      accumulated dJ/d(r0_ord, r0_sup, r0_twin, Q_s, Q_b, b_s, b_b, c, d);
 *   euler_grad         n_grains*3, accumulated dJ/d(phi1, Phi, phi2) per grain (host);
 *   iterations_out     adds the adjoint fixed-point iterations (may be NULL).
 * The handle supplies the material, the load (its strain-controlled components and dt
 * must be those of the increment) and the solver options.  The adjoint fixed point stops
 * on the forward criterion with both relative errors taken against max(|<s>|, |g|_rms)
 * (g the adjoint source); a zero source gives the zero solution without iterating.  It
 * returns RVE_ERR_NOT_CONVERGED after max_iter iterations and RVE_ERR_NAN on a non-finite
 * source or iterate, leaving state_b, eps_b and the gradients unchanged.  The call reuses the
 * handle's spectra: its forward state is lost (keep a copy with rve_save_state).  Needs
 * n_sub <= 16. */
rve_status rve_adjoint_increment(rve_t h, const double* eps_prev, const double* eps_cur, const double* state_prev,
                                 const double dS[6], double dt, double* state_b, double* eps_b, double* param_grad,
                                 double* euler_grad, long long* iterations_out);

/* Effective results.  last (may be NULL) receives the most recent record;
 * hist (may be NULL) receives up to cap records, oldest first; n_hist (may be
 * NULL) receives the number of records held. */
rve_status rve_get_effective(rve_t h, rve_effective* last, rve_effective* hist, int cap,
                             int* n_hist);

/* Copy a committed field into dst (component-major: comp * nvox + voxel) as
 * doubles (dst_bytes must be >= components * nvox * 8).  dst is a host pointer,
 * or a device pointer when dst_on_device. */
rve_status rve_get_fields(rve_t h, int which, void* dst, size_t dst_bytes, int dst_on_device);

/* rve_get_fields with the element type of dst chosen by dtype (rve_dtype):
 * dst_bytes must be >= components * nvox * (8 or 4). */
rve_status rve_get_fields_as(rve_t h, int which, int dtype, void* dst, size_t dst_bytes, int dst_on_device);

/* Checkpoint: rve_save_state with blob == NULL stores the required size in *bytes. */
rve_status rve_save_state(rve_t h, void* blob, size_t* bytes);
rve_status rve_load_state(rve_t h, const void* blob, size_t bytes);

/* Per-kernel device time (CUDA events on the handle's stream) accumulated since the
 * handle was created or last reset, for a handle created with opt.timing != 0.
 * ms[RVE_K_COUNT] receives milliseconds and launches[RVE_K_COUNT] launch counts (either
 * may be NULL); reset != 0 clears the counters after reading.  RVE_ERR_STATE when the
 * handle was created without timing. */
rve_status rve_kernel_times(rve_t h, double* ms, long long* launches, int reset);

/* Convergence history of the most recent increment (committed or not): for each
 * fixed-point iteration i, e_eq[i] = sqrt(sum_xi w |kappa . sigma_hat|^2) / |sigma_hat(0)|
 * (equilibrium error) and c_F[i] = |(<sigma> - Sigma)_F| / |<sigma>| (stress-constraint
 * error).  Up to cap values are written (either array may be NULL); *n receives the
 * number of iterations recorded. */
rve_status rve_get_residuals(rve_t h, double* e_eq, double* c_F, int cap, int* n);

const char* rve_last_error(rve_t h); /* never NULL; h may be NULL (global message) */
void rve_destroy(rve_t h);

/* ---- kernel-level entry points (device pointers, enqueued on `stream`) -------- */

/* Per-voxel constitutive update over one increment (Sec. 3 / Sec. 4, RK4 with n_sub
 * substeps along the linear strain path from eps_n to eps), the hot step of the
 * solver exposed on its own.
 *   R        nvox*9 rotation (row-major, crystal to sample), type by precision;
 *   eps_n    6*nvox strain at t_n; eps 6*nvox strain at t_{n+1} (sample frame);
 *   state    34*nvox crystal-frame state at t_n, updated in place to t_{n+1}:
 *            eps_p (6 comps), v (16), alpha (12), component-major;
 *   sigma    6*nvox output stress at t_{n+1} (sample frame).
 * All arrays are component-major (comp * nvox + voxel) and of the precision's type. */
rve_status rve_material_point(int precision, const rve_material* mat, long long nvox,
                              const void* R, const void* eps_n, const void* eps, void* state,
                              void* sigma, double dt, int n_sub, void* stream);

/* Reverse (vector-Jacobian) pass of rve_material_point: the constitutive building block of
 * the adjoint of a load history (differentiating the Sec. 3 law, the Sec. 4 regularised
 * rates implicitly, and the RK4 substeps).  For given adjoints of the outputs it returns the
 * adjoints of the inputs and of the material parameters.
 *   R, eps_n, eps, state  the forward inputs (as rve_material_point; state at t_n, read only);
 *   sigma_b   6*nvox   adjoint of the stress at t_{n+1};
 *   state_b   34*nvox  in: adjoint of the state at t_{n+1}; out: adjoint of the state at t_n;
 *   eps_b, eps_n_b 6*nvox out: adjoints of eps and eps_n;
 *   R_b       9*nvox   out: adjoint of the rotation entries (component-major, row-major R);
 *   param_b   9*nvox   out: per-voxel adjoints of r0_ord, r0_sup, r0_twin, Q_s, Q_b, b_s,
 *                      b_b, c, d (sum over voxels for the gradient).
 * With sigma_b a unit vector and state_b zero, eps_b is a row of the algorithmic tangent
 * d sigma / d eps.  n_sub <= 16.  Synchronises the stream before returning. */
rve_status rve_material_point_vjp(int precision, const rve_material* mat, long long nvox, const void* R,
                                  const void* eps_n, const void* eps, const void* state, const void* sigma_b,
                                  void* state_b, void* eps_b, void* eps_n_b, void* R_b, void* param_b, double dt,
                                  int n_sub, void* stream);

/* Forward 3-D real-to-complex FFT of ncomp component-major real fields into the
 * solver's half-spectrum layout [comp][kz][ky][kx], kx in [0, nx/2], unnormalised
 * (the transform used in the Green-operator step, Sec. 3).  in: ncomp*nvox reals;
 * out: ncomp*nz*ny*(nx/2+1) complex (interleaved re, im); both device pointers.  Lines of
 * 64, 96, 128, 160 and 256 points take register two-step transforms, other lengths
 * Stockham passes.  The twiddle tables are built on the first call for a (device,
 * precision, length) and kept until the process exits (2 n values each; that first call
 * allocates and copies synchronously); the call synchronises `stream` before returning. */
rve_status rve_fft_r2c(int precision, int nx, int ny, int nz, int ncomp, const void* in,
                       void* out, void* stream);
/* Inverse of rve_fft_r2c, unnormalised (multiply by 1/nvox to invert). The input
 * is overwritten. */
rve_status rve_fft_c2r(int precision, int nx, int ny, int nz, int ncomp, void* in, void* out,
                       void* stream);

/* Periodic Voronoi labelling with the centroid-plane twin split (Sec. 2.1 grains;
 * synthetic twins).  seeds n_parent*3 (x, y, z) in [0,1), twinned n_parent bytes,
 * twin_normal n_parent*3 unit normals (host arrays).  Voxel labels: nearest seed by
 * the squared minimum-image distance of the voxel centre in float64 (ties to the
 * lowest index); a twinned parent p gives id n_parent + p to its voxels on the
 * positive side of the plane through its centroid.  grain_id_out holds nvox labels
 * (host, or device when out_on_device). */
rve_status rve_label_voronoi(int nx, int ny, int nz, int n_parent, const double* seeds,
                             const uint8_t* twinned, const double* twin_normal,
                             uint32_t* grain_id_out, int out_on_device, void* stream);

/* rve_label_voronoi without any device allocation (the paper has no counterpart: this is
 * a service for callers that must not allocate).  Some callers cannot call cudaMalloc or
 * cudaFree: code that owns all device memory through its own pool, code that must not
 * trigger the implicit device-wide synchronisation of those calls (latency-critical
 * loops, other work in flight on the device), and library code embedded where
 * allocation is forbidden.  This variant keeps its scratch (seeds, normals, centroid sums
 * of up to RVE_NOALLOC_MAX_PARENTS parents, about 470 KB) in one static device array that
 * every GPU loading this library holds until the process exits.
 *   Inputs and output as rve_label_voronoi, except that grain_id_out must be a device
 *   pointer (nx*ny*nz labels).  n_parent > RVE_NOALLOC_MAX_PARENTS -> RVE_ERR_INVALID_ARG.
 *   The first call on a device looks up the array's device address (once per device,
 *   with that device current); make that first call before any stream capture.
 *   All calls share the one array: calls whose work overlaps on the GPU (other streams,
 *   other host threads) race and must be serialised by the caller.  The call returns
 *   after its work on `stream` has finished. */
#define RVE_NOALLOC_MAX_PARENTS 4096
rve_status rve_label_voronoi_noalloc(int nx, int ny, int nz, int n_parent, const double* seeds,
                                     const uint8_t* twinned, const double* twin_normal,
                                     uint32_t* grain_id_out, void* stream);

/* ALU throughput probe (the paper has no counterpart: measurement support).  The
 * per-voxel update of rve_material_point is bound by the FP32 (or FP64) FMA pipe and the
 * MUFU unit, so its roofline is taken against rates measured with this probe.
 *   kind     0 FP32 FMA, 1 FP64 FMA, 2 FP32 MUFU ex2.approx;
 *   blocks   CTAs of 256 threads; iters loop trips, each 128 operations per thread
 *            (8 independent chains of 16);
 *   sink     device buffer of at least 8 bytes (written only in a case that does not
 *            occur, so the work is not optimised away);
 *   ops_out  (host, may be NULL) operations of one launch: 2 per FMA, 1 per ex2.
 * Enqueued on `stream` without synchronising; time it with events on that stream. */
rve_status rve_alu_probe(int kind, int blocks, int iters, void* sink, void* stream, double* ops_out);

#ifdef __cplusplus
}
#endif

#endif /* RVE_H */
