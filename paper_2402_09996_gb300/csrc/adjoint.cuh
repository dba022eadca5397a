// Reverse (vector-Jacobian) pass of the per-voxel Meric-Cailletaud update (Sec. 3 law,
// Sec. 4 regularised rates, RK4 substeps along the linear strain path): given adjoints of
// the outputs (stress at t_{n+1} and state at t_{n+1}) it returns adjoints of the inputs
// (strain at t_n and t_{n+1}, state at t_n, rotation) and of the material parameters.
// This is the constitutive building block of the adjoint of the load history; with unit
// stress adjoints it gives the rows of the algorithmic tangent d sigma / d eps.
//
// One forward pass per voxel, with the primal's operations (constitutive.cuh), stores each
// RK4 substep's start state and its four stage rates; every reverse sweep rebuilds a
// stage's intermediates from its input state and stored rates (no rate solve) just
// before reversing it.  The regularised rate rho(a, P) solving rho = P ((a - eta rho)/K)^n is
// differentiated implicitly: with z = (a - eta rho)/K and D = K + eta P n z^(n-1),
//   d rho / d a = P n z^(n-1) / D,   d rho / d P = K z^n / D   (0 where rho = 0).
#pragma once

#include "constitutive.cuh"

namespace rve {

// Adjoints of the material parameters (order of the C ABI's param_bar rows).
constexpr int kParamBar = 9;  // r0_ord, r0_sup, r0_twin, Q_s, Q_b, b_s, b_b, c, d

template <typename T>
struct StageVals {
  T sg[6];
  T ex[16];
  T tek[16];  // slip: tau - c alpha; twins: tau
  T ak[16];
  T rho[16];
  T du_s[6], du_t[6];
  T Es, Et, ftot, wslip, fm_left, Ptw, lg_Ptw;
  T Rb_s, Rb_t;
};

// Forward stage (the operations of rk_stage, one system at a time; the float primal runs
// pairs of systems on packed instructions, which may round the last bit differently):
// rates k of state Y at path point s,
// with the intermediates kept for the reverse pass.  SOLVE = false takes the rates rho of
// the 16 systems from rho_in (a stage evaluated before with the same Y and s) instead of
// solving for them, and rebuilds everything else.
template <typename T, int NP, bool SOLVE = true>
__device__ __forceinline__ void stage_eval(const MatDev<T>& M, const T* e0, const T* de, T s, const MPState<T>& Y,
                                           const T* tab, StageVals<T>& V, MPState<T>& k,
                                           const T* rho_in = nullptr) {
  constexpr double kLog2e = 1.44269504088896340736;
  T e[6];
  #pragma unroll
  for (int c = 0; c < 6; ++c) e[c] = e0[c] + s * de[c] - Y.ep[c];
  hooke<T>(M, e, V.sg);
  V.Es = T(0);
  V.Et = T(0);
  T vtw = T(0);
  const T cb_s = -M.b_s * T(kLog2e), cb_t = -M.b_b * T(kLog2e);
  #pragma unroll
  for (int q = 0; q < 12; ++q) {
    V.ex[q] = fast_exp2<T>(cb_s * Y.v[q]);
    V.Es += V.ex[q];
  }
  #pragma unroll
  for (int q = 12; q < 16; ++q) {
    V.ex[q] = fast_exp2<T>(cb_t * Y.v[q]);
    V.Et += V.ex[q];
    vtw += Y.v[q];
  }
  V.ftot = T(1.41421356237309504880) * vtw;
  V.wslip = T(1) - V.ftot;
  V.fm_left = M.fm - V.ftot;
  V.fm_left = V.fm_left > T(0) ? V.fm_left : T(0);
  V.Ptw = (M.Kc * T(0.70710678118654752440)) * V.fm_left;
  V.lg_Ptw = fast_log2<T>(V.Ptw > T(0) ? V.Ptw : T(1));
  const T dq = M.h_diag - M.h_off;
  const T Qdq_s = M.Q_s * dq, Qdq_t = M.Q_b * dq;
  V.Rb_s = M.Q_s * (M.h_off * (T(12) - V.Es) + dq);
  V.Rb_t = M.Q_b * (M.h_off * (T(4) - V.Et) + dq);
  RootCoef<T> qs, qt;
  if constexpr (NP != 0 && SOLVE) {
    qs = root_coef<T>(T(1), M.K, M.n, M.inv_n, M.lg_K, M.eta, M.lg_eta, T(0));
    qt = root_coef<T>(V.Ptw, M.Kt, M.nt, M.inv_nt, M.lg_Kt, M.eta, M.lg_eta, V.lg_Ptw);
  }
  T ss[6];
  #pragma unroll
  for (int c = 0; c < 6; ++c) ss[c] = V.sg[c] * sys_scale<T>(0);
  #pragma unroll
  for (int c = 0; c < 6; ++c) V.du_s[c] = V.du_t[c] = T(0);
  #pragma unroll
  for (int q = 0; q < 12; ++q) {
    V.tek[q] = schmid_sum<T>(q, ss) - M.c * Y.al[q];
    V.ak[q] = fabs(V.tek[q]) - ((M.r0[q] + V.Rb_s) - Qdq_s * V.ex[q]);
    if constexpr (SOLVE) V.rho[q] = stage_rate<T, NP>(M, qs, V.ak[q], T(1), false, T(0), tab);
    else V.rho[q] = rho_in[q];
    const T gd = copysign(V.rho[q], V.tek[q]);
    schmid_add<T>(q, gd, V.du_s);
    k.v[q] = V.rho[q];
    k.al[q] = gd - M.d * V.rho[q] * Y.al[q];
  }
  #pragma unroll
  for (int q = 12; q < 16; ++q) {
    V.tek[q] = sys_scale<T>(q) * schmid_sum<T>(q, V.sg);
    V.ak[q] = V.tek[q] - ((M.r0[q] + V.Rb_t) - Qdq_t * V.ex[q]);
    if constexpr (SOLVE) V.rho[q] = stage_rate<T, NP>(M, qt, V.ak[q], V.Ptw, true, V.lg_Ptw, tab);
    else V.rho[q] = rho_in[q];
    schmid_add<T>(q, V.rho[q], V.du_t);
    k.v[q] = V.rho[q];
  }
  const T fs = V.wslip * sys_scale<T>(0);
  #pragma unroll
  for (int c = 0; c < 6; ++c) {
    const T wc = c < 3 ? T(1) : T(0.5);
    k.ep[c] = wc * (fs * V.du_s[c] + sys_scale<T>(12) * V.du_t[c]);
  }
}

// d rho / d a and d rho / d P at a solved root (rho, a, P; exponent n, K, eta).
template <typename T>
__device__ void root_partials(T rho, T a, T P, T Kn, T n, T eta, T* d_a, T* d_P) {
  if (!(rho > T(0)) || !(P > T(0))) {
    *d_a = T(0);
    *d_P = T(0);
    return;
  }
  const T z = (a - eta * rho) / Kn;
  if (!(z > T(0))) {
    *d_a = T(0);
    *d_P = T(0);
    return;
  }
  const T zn = rho / P;              // z^n
  const T pnz = P * n * (zn / z);    // P n z^(n-1)
  const T D = Kn + eta * pnz;
  *d_a = pnz / D;
  *d_P = Kn * zn / D;
}

// Reverse of stage_eval: kb = adjoint of the rates; adds the adjoints of Y, e0, de and
// the parameters.
template <typename T>
__device__ void stage_vjp(const MatDev<T>& M, const T* de, T s, const MPState<T>& Y, const StageVals<T>& V,
                          const MPState<T>& kb, MPState<T>& Yb, T* e0b, T* deb, T* pb) {
  constexpr double kLog2e = 1.44269504088896340736;
  (void)kLog2e;
  (void)de;
  const T dq = M.h_diag - M.h_off;
  const T ssc = sys_scale<T>(0), tsc = sys_scale<T>(12);
  // eps_p rate: k.ep[c] = wc (wslip ssc du_s[c] + tsc du_t[c])
  T dusb[6], dutb[6];
  T wslipb = T(0);
  #pragma unroll
  for (int c = 0; c < 6; ++c) {
    const T wc = c < 3 ? T(1) : T(0.5);
    dusb[c] = kb.ep[c] * wc * V.wslip * ssc;
    dutb[c] = kb.ep[c] * wc * tsc;
    wslipb += kb.ep[c] * wc * ssc * V.du_s[c];
  }
  T sgb[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  T exb[16];
  #pragma unroll
  for (int q = 0; q < 16; ++q) exb[q] = T(0);
  T Esb = T(0), Etb = T(0), Ptwb = T(0);
  // slip systems
  #pragma unroll
  for (int q = 0; q < 12; ++q) {
    const T sgn = V.tek[q] < T(0) ? T(-1) : T(1);
    const T gd = sgn * V.rho[q];
    // gd enters du_s (schmid_add) and k.al = gd - d rho al
    T gdb = kb.al[q];
    #pragma unroll
    for (int c = 0; c < 6; ++c) gdb += T(schmid_k(q, c)) * dusb[c];
    T rhob = kb.v[q] + sgn * gdb - M.d * Y.al[q] * kb.al[q];
    Yb.al[q] += -M.d * V.rho[q] * kb.al[q];
    pb[8] += -V.rho[q] * Y.al[q] * kb.al[q];  // d
    (void)gd;
    T d_a, d_P;
    root_partials<T>(V.rho[q], V.ak[q], T(1), M.K, M.n, M.eta, &d_a, &d_P);
    const T akb = rhob * d_a;
    // a = |tek| - ((r0 + Rb_s) - Qdq_s ex)
    const T tekb = akb * sgn;
    const T rb = -akb;
    pb[(q % 3 == 2) ? 0 : 1] += rb;  // r0: ordinary systems 2, 5, 8, 11; the rest superdislocations
    Esb += rb * (-M.Q_s * M.h_off);
    exb[q] += rb * (-M.Q_s * dq);
    pb[3] += rb * ((M.h_off * (T(12) - V.Es) + dq) - dq * V.ex[q]);  // Q_s
    // tek = ssc sum K sg - c al
    Yb.al[q] += -M.c * tekb;
    pb[7] += -Y.al[q] * tekb;  // c
    #pragma unroll
    for (int c = 0; c < 6; ++c) sgb[c] += ssc * T(schmid_k(q, c)) * tekb;
  }
  // twins
  #pragma unroll
  for (int q = 12; q < 16; ++q) {
    T rhob = kb.v[q];
    #pragma unroll
    for (int c = 0; c < 6; ++c) rhob += T(schmid_k(q, c)) * dutb[c];
    T d_a, d_P;
    root_partials<T>(V.rho[q], V.ak[q], V.Ptw, M.Kt, M.nt, M.eta, &d_a, &d_P);
    const T akb = rhob * d_a;
    Ptwb += rhob * d_P;
    const T rb = -akb;
    pb[2] += rb;  // r0_twin
    Etb += rb * (-M.Q_b * M.h_off);
    exb[q] += rb * (-M.Q_b * dq);
    pb[4] += rb * ((M.h_off * (T(4) - V.Et) + dq) - dq * V.ex[q]);  // Q_b
    #pragma unroll
    for (int c = 0; c < 6; ++c) sgb[c] += tsc * T(schmid_k(q, c)) * akb;
  }
  // Ptw = Kc/sqrt2 max(fm - ftot, 0); wslip = 1 - ftot; ftot = sqrt2 sum v_twin
  T ftotb = -wslipb;
  if (V.fm_left > T(0)) ftotb += Ptwb * (-(M.Kc * T(0.70710678118654752440)));
  const T vtwb = T(1.41421356237309504880) * ftotb;
  // ex = exp(-b v)
  #pragma unroll
  for (int q = 0; q < 12; ++q) {
    exb[q] += Esb;
    Yb.v[q] += exb[q] * (-M.b_s * V.ex[q]);
    pb[5] += exb[q] * (-Y.v[q] * V.ex[q]);  // b_s
  }
  #pragma unroll
  for (int q = 12; q < 16; ++q) {
    exb[q] += Etb;
    Yb.v[q] += exb[q] * (-M.b_b * V.ex[q]) + vtwb;
    pb[6] += exb[q] * (-Y.v[q] * V.ex[q]);  // b_b
  }
  // sg = hooke(e), e = e0 + s de - ep
  T eb[6];
  eb[0] = M.C11 * sgb[0] + M.C12 * sgb[1] + M.C13 * sgb[2];
  eb[1] = M.C12 * sgb[0] + M.C11 * sgb[1] + M.C13 * sgb[2];
  eb[2] = M.C13 * (sgb[0] + sgb[1]) + M.C33 * sgb[2];
  eb[3] = T(2) * M.C44 * sgb[3];
  eb[4] = T(2) * M.C44 * sgb[4];
  eb[5] = T(2) * M.C66 * sgb[5];
  #pragma unroll
  for (int c = 0; c < 6; ++c) {
    e0b[c] += eb[c];
    deb[c] += s * eb[c];
    Yb.ep[c] -= eb[c];
  }
}

// Symmetric 3x3 from 6 components (11 22 33 23 13 12) and back.
template <typename T>
__device__ __forceinline__ void sym33(const T* v, T A[3][3]) {
  A[0][0] = v[0]; A[1][1] = v[1]; A[2][2] = v[2];
  A[1][2] = A[2][1] = v[3];
  A[0][2] = A[2][0] = v[4];
  A[0][1] = A[1][0] = v[5];
}
// adjoint of `sym33` for a symmetric tensor adjoint G: off-diagonal components appear twice
template <typename T>
__device__ __forceinline__ void sym33_adj(const T G[3][3], T* vb) {
  vb[0] = G[0][0]; vb[1] = G[1][1]; vb[2] = G[2][2];
  vb[3] = G[1][2] + G[2][1];
  vb[4] = G[0][2] + G[2][0];
  vb[5] = G[0][1] + G[1][0];
}
// tensor adjoint of a 6-component output taken from a symmetric tensor (one entry each)
template <typename T>
__device__ __forceinline__ void out6_adj(const T* ob, T G[3][3]) {
  G[0][0] = ob[0]; G[1][1] = ob[1]; G[2][2] = ob[2];
  G[1][2] = G[2][1] = T(0.5) * ob[3];
  G[0][2] = G[2][0] = T(0.5) * ob[4];
  G[0][1] = G[1][0] = T(0.5) * ob[5];
}

// out = R^T E R (to_crystal): given out_b, adds E_b (6) and R_b (9).
template <typename T>
__device__ void to_crystal_vjp(const T* R, const T* e, const T* ob, T* eb, T* Rb) {
  T G[3][3], E[3][3];
  out6_adj<T>(ob, G);
  sym33<T>(e, E);
  // E_b = R G R^T ; R_b = 2 E R G
  T Eb[3][3];
  #pragma unroll
  for (int i = 0; i < 3; ++i)
    #pragma unroll
    for (int j = 0; j < 3; ++j) {
      T acc = T(0);
      #pragma unroll
      for (int a = 0; a < 3; ++a)
        #pragma unroll
        for (int b = 0; b < 3; ++b) acc += R[i * 3 + a] * G[a][b] * R[j * 3 + b];
      Eb[i][j] = acc;
    }
  T eb6[6];
  sym33_adj<T>(Eb, eb6);
  #pragma unroll
  for (int c = 0; c < 6; ++c) eb[c] += eb6[c];
  #pragma unroll
  for (int i = 0; i < 3; ++i)
    #pragma unroll
    for (int j = 0; j < 3; ++j) {
      T acc = T(0);
      #pragma unroll
      for (int a = 0; a < 3; ++a)
        #pragma unroll
        for (int b = 0; b < 3; ++b) acc += E[i][a] * R[a * 3 + b] * G[b][j];
      Rb[i * 3 + j] += T(2) * acc;
    }
}

// out = R S R^T (to_sample): given out_b, adds S_b (6) and R_b (9).
template <typename T>
__device__ void to_sample_vjp(const T* R, const T* s, const T* ob, T* sb, T* Rb) {
  T G[3][3], S[3][3];
  out6_adj<T>(ob, G);
  sym33<T>(s, S);
  T Sb[3][3];
  #pragma unroll
  for (int i = 0; i < 3; ++i)
    #pragma unroll
    for (int j = 0; j < 3; ++j) {
      T acc = T(0);
      #pragma unroll
      for (int a = 0; a < 3; ++a)
        #pragma unroll
        for (int b = 0; b < 3; ++b) acc += R[a * 3 + i] * G[a][b] * R[b * 3 + j];
      Sb[i][j] = acc;
    }
  T sb6[6];
  sym33_adj<T>(Sb, sb6);
  #pragma unroll
  for (int c = 0; c < 6; ++c) sb[c] += sb6[c];
  #pragma unroll
  for (int i = 0; i < 3; ++i)
    #pragma unroll
    for (int j = 0; j < 3; ++j) {
      T acc = T(0);
      #pragma unroll
      for (int a = 0; a < 3; ++a)
        #pragma unroll
        for (int b = 0; b < 3; ++b) acc += G[i][a] * R[a * 3 + b] * S[b][j];
      Rb[i * 3 + j] += T(2) * acc;
    }
}

template <typename T>
__device__ __forceinline__ void state_axpy(MPState<T>& y, T w, const MPState<T>& x) {
  #pragma unroll
  for (int c = 0; c < 6; ++c) y.ep[c] += w * x.ep[c];
  #pragma unroll
  for (int c = 0; c < 16; ++c) y.v[c] += w * x.v[c];
  #pragma unroll
  for (int c = 0; c < 12; ++c) y.al[c] += w * x.al[c];
}
template <typename T>
__device__ __forceinline__ void state_zero(MPState<T>& y) {
  #pragma unroll
  for (int c = 0; c < 6; ++c) y.ep[c] = T(0);
  #pragma unroll
  for (int c = 0; c < 16; ++c) y.v[c] = T(0);
  #pragma unroll
  for (int c = 0; c < 12; ++c) y.al[c] = T(0);
}


// Forward pass of mc_voxel that keeps what the reverse sweeps need: the start state of
// every RK4 substep (ys[0..nsub]) and the rates of its four stages (ks[4 m + j]).  The
// update arithmetic is the primal's (classical RK4, weights 1 2 2 1, stage inputs
// y + h/2 k1, y + h/2 k2, y + h k3).
template <typename T, int NP>
__device__ __forceinline__ void mc_forward_store(const MatDev<T>& M, const T* e0, const T* de, T dt, int nsub,
                                                 const T* tab, MPState<T>* ys, MPState<T>* ks) {
  const T h = dt / T(nsub);
  const T inv = T(1) / T(nsub);
  StageVals<T> V;
#pragma unroll 1
  for (int m = 0; m < nsub; ++m) {
    const T s0 = T(m) * inv, sh = (T(m) + T(0.5)) * inv, s1 = (T(m) + T(1)) * inv;
    MPState<T> k, Y, acc;
    state_zero<T>(acc);
    stage_eval<T, NP>(M, e0, de, s0, ys[m], tab, V, k);
    ks[4 * m] = k;
    state_axpy<T>(acc, T(1), k);
    Y = ys[m];
    state_axpy<T>(Y, T(0.5) * h, k);
    stage_eval<T, NP>(M, e0, de, sh, Y, tab, V, k);
    ks[4 * m + 1] = k;
    state_axpy<T>(acc, T(2), k);
    Y = ys[m];
    state_axpy<T>(Y, T(0.5) * h, k);
    stage_eval<T, NP>(M, e0, de, sh, Y, tab, V, k);
    ks[4 * m + 2] = k;
    state_axpy<T>(acc, T(2), k);
    Y = ys[m];
    state_axpy<T>(Y, h, k);
    stage_eval<T, NP>(M, e0, de, s1, Y, tab, V, k);
    ks[4 * m + 3] = k;
    state_axpy<T>(acc, T(1), k);
    Y = ys[m];
    state_axpy<T>(Y, h / T(6), acc);
    ys[m + 1] = Y;
  }
}

// Reverse sweep of mc_voxel over a stored forward pass (mc_forward_store; quiet: the
// increment was elastic, ys[nsub] = ys[0]).  In: sigma_b (adjoint of the stress at t_{n+1}),
// yb (adjoint of the state at t_{n+1}; overwritten with the adjoint of the state at t_n).
// Out (added): eps_nb, epsb, Rb, pb (kParamBar).  Each stage is rebuilt from its stored
// input state and rates (no rate solve) just before it is reversed.
template <typename T, int NP>
__device__ __forceinline__ void mc_reverse(const MatDev<T>& M, const T* R, const T* eps_n, const T* eps,
                                           const T* e0, const T* e1, const T* de, bool quiet,
                                           const MPState<T>* ys, const MPState<T>* ks, T dt, int nsub,
                                           const T* sigma_b, MPState<T>& yb, T* eps_nb, T* epsb, T* Rb, T* pb,
                                           const T* tab) {
  const MPState<T>& yN = ys[quiet ? 0 : nsub];
  // stress: sc = C (e1 - ep_N); sigma = R sc R^T
  T ee[6], sc[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) ee[c] = e1[c] - yN.ep[c];
  hooke<T>(M, ee, sc);
  T scb[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  to_sample_vjp<T>(R, sc, sigma_b, scb, Rb);
  T eeb[6];
  eeb[0] = M.C11 * scb[0] + M.C12 * scb[1] + M.C13 * scb[2];
  eeb[1] = M.C12 * scb[0] + M.C11 * scb[1] + M.C13 * scb[2];
  eeb[2] = M.C13 * (scb[0] + scb[1]) + M.C33 * scb[2];
  eeb[3] = T(2) * M.C44 * scb[3];
  eeb[4] = T(2) * M.C44 * scb[4];
  eeb[5] = T(2) * M.C66 * scb[5];
  T e0b[6], e1b[6], deb[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    e1b[c] = eeb[c];
    yb.ep[c] -= eeb[c];
    e0b[c] = T(0);
    deb[c] = T(0);
  }
  if (!quiet) {
    const T h = dt / T(nsub);
    const T inv = T(1) / T(nsub);
#pragma unroll 1
    for (int m = nsub - 1; m >= 0; --m) {
      const T s0 = T(m) * inv, sh = (T(m) + T(0.5)) * inv, s1 = (T(m) + T(1)) * inv;
      // y' = y + h/6 (k1 + 2 k2 + 2 k3 + k4); yend = adjoint of y'
      const MPState<T> yend = yb;
      MPState<T> Y, kb, Yb, kdum;
      StageVals<T> V;
      // stage 4 at Y4 = y + h k3
      Y = ys[m];
      state_axpy<T>(Y, h, ks[4 * m + 2]);
      stage_eval<T, NP, false>(M, e0, de, s1, Y, tab, V, kdum, ks[4 * m + 3].v);
      state_zero<T>(kb);
      state_axpy<T>(kb, h / T(6), yend);
      state_zero<T>(Yb);
      stage_vjp<T>(M, de, s1, Y, V, kb, Yb, e0b, deb, pb);
      state_axpy<T>(yb, T(1), Yb);
      // stage 3 at Y3 = y + h/2 k2; k3 feeds y' and Y4
      state_zero<T>(kb);
      state_axpy<T>(kb, h / T(3), yend);
      state_axpy<T>(kb, h, Yb);
      Y = ys[m];
      state_axpy<T>(Y, T(0.5) * h, ks[4 * m + 1]);
      stage_eval<T, NP, false>(M, e0, de, sh, Y, tab, V, kdum, ks[4 * m + 2].v);
      state_zero<T>(Yb);
      stage_vjp<T>(M, de, sh, Y, V, kb, Yb, e0b, deb, pb);
      state_axpy<T>(yb, T(1), Yb);
      // stage 2 at Y2 = y + h/2 k1; k2 feeds y' and Y3
      state_zero<T>(kb);
      state_axpy<T>(kb, h / T(3), yend);
      state_axpy<T>(kb, T(0.5) * h, Yb);
      Y = ys[m];
      state_axpy<T>(Y, T(0.5) * h, ks[4 * m]);
      stage_eval<T, NP, false>(M, e0, de, sh, Y, tab, V, kdum, ks[4 * m + 1].v);
      state_zero<T>(Yb);
      stage_vjp<T>(M, de, sh, Y, V, kb, Yb, e0b, deb, pb);
      state_axpy<T>(yb, T(1), Yb);
      // stage 1 at y; k1 feeds y' and Y2
      state_zero<T>(kb);
      state_axpy<T>(kb, h / T(6), yend);
      state_axpy<T>(kb, T(0.5) * h, Yb);
      stage_eval<T, NP, false>(M, e0, de, s0, ys[m], tab, V, kdum, ks[4 * m].v);
      state_zero<T>(Yb);
      stage_vjp<T>(M, de, s0, ys[m], V, kb, Yb, e0b, deb, pb);
      state_axpy<T>(yb, T(1), Yb);
    }
  }
  // de = e1 - e0; e0 = R^T eps_n R; e1 = R^T eps R
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    e1b[c] += deb[c];
    e0b[c] -= deb[c];
  }
  to_crystal_vjp<T>(R, eps_n, e0b, eps_nb, Rb);
  to_crystal_vjp<T>(R, eps, e1b, epsb, Rb);
}

// Per-voxel inputs of the reverse kernels: rotation, strains (sample frame), state at t_n,
// and the stored forward pass.
template <typename T>
struct VjpVoxel {
  T r[9], en[6], e[6], e0[6], e1[6], de[6];
  MPState<T> ys[kMaxSubVjp + 1];
  MPState<T> ks[4 * kMaxSubVjp];
  bool quiet;
};

template <typename T, int NP>
__device__ __forceinline__ void vjp_prepare(const MatDev<T>& M, long long i, size_t n, const T* __restrict__ R,
                                            const T* __restrict__ eps_n, const T* __restrict__ eps,
                                            const T* __restrict__ state, T dt, int nsub, const T* tab,
                                            VjpVoxel<T>& P) {
#pragma unroll
  for (int k = 0; k < 9; ++k) P.r[k] = R[(size_t)i * 9 + k];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    P.en[c] = eps_n[c * n + i];
    P.e[c] = eps[c * n + i];
  }
  MPState<T> y;
#pragma unroll
  for (int c = 0; c < 6; ++c) y.ep[c] = state[c * n + i];
#pragma unroll
  for (int c = 0; c < 16; ++c) y.v[c] = state[(6 + c) * n + i];
#pragma unroll
  for (int c = 0; c < 12; ++c) y.al[c] = state[(22 + c) * n + i];
  to_crystal<T>(P.r, P.en, P.e0);
  to_crystal<T>(P.r, P.e, P.e1);
#pragma unroll
  for (int c = 0; c < 6; ++c) P.de[c] = P.e1[c] - P.e0[c];
  P.quiet = elastic_increment<T>(M, P.e0, P.de, y);
  P.ys[0] = y;
  if (!P.quiet) mc_forward_store<T, NP>(M, P.e0, P.de, dt, nsub, tab, P.ys, P.ks);
}

template <typename T>
__device__ __forceinline__ void load_state34(const T* __restrict__ src, long long i, size_t n, MPState<T>& y) {
#pragma unroll
  for (int c = 0; c < 6; ++c) y.ep[c] = src[c * n + i];
#pragma unroll
  for (int c = 0; c < 16; ++c) y.v[c] = src[(6 + c) * n + i];
#pragma unroll
  for (int c = 0; c < 12; ++c) y.al[c] = src[(22 + c) * n + i];
}
template <typename T>
__device__ __forceinline__ void store_state34(T* __restrict__ dst, long long i, size_t n, const MPState<T>& y) {
#pragma unroll
  for (int c = 0; c < 6; ++c) dst[c * n + i] = y.ep[c];
#pragma unroll
  for (int c = 0; c < 16; ++c) dst[(6 + c) * n + i] = y.v[c];
#pragma unroll
  for (int c = 0; c < 12; ++c) dst[(22 + c) * n + i] = y.al[c];
}

// One thread per voxel; arrays component-major (component * nvox + voxel) as in the
// forward material-point kernel.  state_b: in, adjoint of the state at t_{n+1}; out, adjoint
// of the state at t_n.  R_b (9 x nvox) and param_b (kParamBar x nvox) are per voxel.
template <typename T, int NP>
__global__ void k_material_point_vjp(const MatDev<T> M, long long nvox, const T* __restrict__ R,
                                     const T* __restrict__ eps_n, const T* __restrict__ eps,
                                     const T* __restrict__ state, T dt, int nsub, const T* __restrict__ sigma_b,
                                     T* state_b, T* eps_b, T* eps_n_b, T* R_b, T* param_b,
                                     const T* __restrict__ root_tab) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw);
  if (NP != 0)
    for (int k = threadIdx.x; k < kRootTabs; k += blockDim.x) tab[k] = root_tab[k];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvox) return;
  const size_t n = (size_t)nvox;
  VjpVoxel<T> P;
  vjp_prepare<T, NP>(M, i, n, R, eps_n, eps, state, dt, nsub, tab, P);
  T sb[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) sb[c] = sigma_b[c * n + i];
  MPState<T> yb;
  load_state34<T>(state_b, i, n, yb);
  T enb[6] = {T(0), T(0), T(0), T(0), T(0), T(0)}, eb[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  T rb[9] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  T pb[kParamBar];
#pragma unroll
  for (int k = 0; k < kParamBar; ++k) pb[k] = T(0);
  mc_reverse<T, NP>(M, P.r, P.en, P.e, P.e0, P.e1, P.de, P.quiet, P.ys, P.ks, dt, nsub, sb, yb, enb, eb, rb, pb, tab);
  store_state34<T>(state_b, i, n, yb);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    eps_b[c * n + i] = eb[c];
    eps_n_b[c * n + i] = enb[c];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) R_b[k * n + i] = rb[k];
#pragma unroll
  for (int k = 0; k < kParamBar; ++k) param_b[k * n + i] = pb[k];
}

// The reverse work of one increment of the history adjoint before its fixed point, over one
// stored forward pass per voxel: the six rows J(k, .) = d sigma_k / d eps of the algorithmic
// tangent (unit stress adjoints, no state adjoint; written to J at (k * 6 + c) * nvox + voxel)
// and the direct part (uniform stress adjoint sd, state adjoint state_b at t_{n+1}, which is
// overwritten with the adjoint at t_n), whose eps, eps_n, rotation and parameter adjoints go
// to eps_b, eps_n_b, R_b and param_b.
template <typename T, int NP>
__global__ void k_adj_tangent(const MatDev<T> M, long long nvox, const T* __restrict__ R,
                              const T* __restrict__ eps_n, const T* __restrict__ eps,
                              const T* __restrict__ state, T dt, int nsub, T sd0, T sd1, T sd2, T sd3, T sd4, T sd5,
                              T* state_b, T* J, T* eps_b, T* eps_n_b, T* R_b, T* param_b,
                              const T* __restrict__ root_tab) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw);
  if (NP != 0)
    for (int k = threadIdx.x; k < kRootTabs; k += blockDim.x) tab[k] = root_tab[k];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvox) return;
  const size_t n = (size_t)nvox;
  VjpVoxel<T> P;
  vjp_prepare<T, NP>(M, i, n, R, eps_n, eps, state, dt, nsub, tab, P);
#pragma unroll 1
  for (int row = 0; row < 7; ++row) {
    T sb[6];
    MPState<T> yb;
    if (row < 6) {
#pragma unroll
      for (int c = 0; c < 6; ++c) sb[c] = c == row ? T(1) : T(0);
      state_zero<T>(yb);
    } else {
      sb[0] = sd0; sb[1] = sd1; sb[2] = sd2; sb[3] = sd3; sb[4] = sd4; sb[5] = sd5;
      load_state34<T>(state_b, i, n, yb);
    }
    T enb[6] = {T(0), T(0), T(0), T(0), T(0), T(0)}, eb[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T rb[9] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    T pb[kParamBar];
#pragma unroll
    for (int k = 0; k < kParamBar; ++k) pb[k] = T(0);
    mc_reverse<T, NP>(M, P.r, P.en, P.e, P.e0, P.e1, P.de, P.quiet, P.ys, P.ks, dt, nsub, sb, yb, enb, eb, rb, pb,
                      tab);
    if (row < 6) {
#pragma unroll
      for (int c = 0; c < 6; ++c) J[((size_t)row * 6 + c) * n + i] = eb[c];
    } else {
      store_state34<T>(state_b, i, n, yb);
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        eps_b[c * n + i] = eb[c];
        eps_n_b[c * n + i] = enb[c];
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) R_b[k * n + i] = rb[k];
#pragma unroll
      for (int k = 0; k < kParamBar; ++k) param_b[k * n + i] = pb[k];
    }
  }
}

}  // namespace rve
