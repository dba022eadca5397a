"""FP64 CPU oracle: FFT Green-operator fixed point + Meric-Cailletaud crystal plasticity.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline leg import this module; the library never does, and this module
imports nothing from the library.

It restates, in plain numpy float64 with tensors kept as 3x3 arrays, the method
of arXiv 2402.09996:

* Sec. 3, small-strain split and Hooke's law sigma = C : (eps - eps_p);
* Sec. 3, Eq. for the plastic strain rate (twin-fraction weighted sum of slip and
  pseudo-slip), the Schmid tensor m = (n x l + l x n)/2, the resolved shear
  tau = sigma : m, isotropic hardening with an interaction matrix, Norton flow for
  slip and the unidirectional twin law with f = sqrt(2) v;
* Table 1 for the 12 slip and 4 twin systems;
* Sec. 4, Eq. (regu): the viscous regularisation r' = r + eta |gamma_dot|, solved at
  the same instant as the rate (the paper leaves the instant open);
* Sec. 3 (end): explicit RK4 integration per voxel, coupled to a Green-operator
  ("FFT") solver -- here the basic fixed-point scheme with Willot's rotated
  discrete Green operator (the paper names no discretisation) and a mixed macroscopic
  load (strain rate on the controlled components, zero mean stress on the others).

Nothing here is blocked, fused or reordered for speed.  Parity status of each
function is stated in its docstring; all are pinned by tests/test_oracle_*.py.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SQRT2 = math.sqrt(2.0)

# ----------------------------------------------------------------------------------
# Table 1: slip planes n and directions l (crystal frame, Miller indices, c/a = 1).
# System 9 is read as (1 -1 1)[1 1 0]: Table 1 prints [0 1 1], a duplicate of system 7.
# ----------------------------------------------------------------------------------
SLIP_TABLE = [
    # (plane, direction, kind)  kind: "s" superdislocation, "o" ordinary dislocation
    ((1, 1, -1), (0, 1, 1), "s"),
    ((1, 1, -1), (1, 0, 1), "s"),
    ((1, 1, -1), (1, -1, 0), "o"),
    ((-1, 1, 1), (0, -1, 1), "s"),
    ((-1, 1, 1), (-1, 0, -1), "s"),
    ((-1, 1, 1), (-1, -1, 0), "o"),
    ((1, -1, 1), (0, 1, 1), "s"),
    ((1, -1, 1), (1, 0, -1), "s"),
    ((1, -1, 1), (1, 1, 0), "o"),
    ((1, 1, 1), (0, 1, -1), "s"),
    ((1, 1, 1), (1, 0, -1), "s"),
    ((1, 1, 1), (1, -1, 0), "o"),
]
TWIN_TABLE = [
    ((1, 1, -1), (1, 1, 2)),
    ((-1, 1, 1), (-1, 1, -2)),
    ((1, -1, 1), (1, -1, -2)),
    ((1, 1, 1), (1, 1, -2)),
]
N_SLIP = 12
N_TWIN = 4
N_SYS = N_SLIP + N_TWIN


def system_vectors():
    """Unit plane normals and slip directions of the 16 systems (Table 1; lattice read as pseudo-cubic, c/a = 1).

    Returns (n, l, kinds): arrays (16, 3) and a list of 16 kinds ("s", "o", "t").
    Parity: pinned (tests/test_oracle_tables.py: orthogonality, Schmid factors).
    """
    n = np.array([p for p, _, _ in SLIP_TABLE] + [p for p, _ in TWIN_TABLE], dtype=np.float64)
    l = np.array([d for _, d, _ in SLIP_TABLE] + [d for _, d in TWIN_TABLE], dtype=np.float64)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    l /= np.linalg.norm(l, axis=1, keepdims=True)
    kinds = [k for _, _, k in SLIP_TABLE] + ["t"] * N_TWIN
    return n, l, kinds


def schmid_tensors():
    """m = (n x l + l x n) / 2 for the 16 systems (Sec. 3, Schmid tensor). Shape (16, 3, 3)."""
    n, l, _ = system_vectors()
    return 0.5 * (n[:, :, None] * l[:, None, :] + l[:, :, None] * n[:, None, :])


# ----------------------------------------------------------------------------------
# Material
# ----------------------------------------------------------------------------------
@dataclass
class Material:
    """Constants of Sec. 3 / Sec. 4 (MPa, s).  Defaults: the 16^3 and 128^3 workloads.

    Elastic moduli and the twin constants Kc, fm and eta follow the paper
    (C33 = 178 GPa as in the workload description); r0, K, n, Q, b, the interaction
    matrix and the kinematic constants c, d follow the workload description.
    """

    C11: float = 183000.0
    C12: float = 74000.0
    C13: float = 74000.0
    C33: float = 178000.0
    C44: float = 105000.0
    C66: float = 78000.0
    r0_ord: float = 90.0
    r0_sup: float = 200.0
    r0_twin: float = 110.0
    K: float = 10.0
    n: float = 10.0
    Kt: float = 10.0
    nt: float = 10.0
    Q_s: float = 20.0
    Q_b: float = 20.0
    b_s: float = 5.0
    b_b: float = 5.0
    h_diag: float = 1.0
    h_off: float = 1.2
    c: float = 10000.0
    d: float = 500.0
    Kc: float = 1.45
    fm: float = 0.8
    eta: float = 1.0e4

    def r0_vector(self):
        _, _, kinds = system_vectors()
        table = {"o": self.r0_ord, "s": self.r0_sup, "t": self.r0_twin}
        return np.array([table[k] for k in kinds])


def stiffness_tensor(mat: Material) -> np.ndarray:
    """Tetragonal stiffness C_ijkl (crystal c axis = z) from c11, c12, c13, c33, c44, c66.

    Sec. 3, elastic moduli.  Built from the 6x6 Voigt matrix with every minor-symmetric
    index placement.  Parity: pinned (uniaxial modulus closed form, laminate).
    """
    V = np.zeros((6, 6))
    V[0, 0] = V[1, 1] = mat.C11
    V[2, 2] = mat.C33
    V[0, 1] = V[1, 0] = mat.C12
    V[0, 2] = V[2, 0] = V[1, 2] = V[2, 1] = mat.C13
    V[3, 3] = V[4, 4] = mat.C44
    V[5, 5] = mat.C66
    pair = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (1, 2): 3, (2, 1): 3, (0, 2): 4, (2, 0): 4, (0, 1): 5, (1, 0): 5}
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C[i, j, k, l] = V[pair[(i, j)], pair[(k, l)]]
    return C


def isotropic_tensor(lam: float, mu: float) -> np.ndarray:
    """C0_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk)."""
    d = np.eye(3)
    return lam * np.einsum("ij,kl->ijkl", d, d) + mu * (
        np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)
    )


# Mandel map: (11, 22, 33, 23, 13, 12) with sqrt(2) on shears (an isometry).
_MANDEL_IDX = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
_MANDEL_W = np.array([1.0, 1.0, 1.0, SQRT2, SQRT2, SQRT2])


def to_mandel(t: np.ndarray) -> np.ndarray:
    return np.stack([t[..., i, j] for i, j in _MANDEL_IDX], axis=-1) * _MANDEL_W


def from_mandel(v: np.ndarray) -> np.ndarray:
    out = np.zeros(v.shape[:-1] + (3, 3), dtype=v.dtype)
    for a, (i, j) in enumerate(_MANDEL_IDX):
        out[..., i, j] = v[..., a] / _MANDEL_W[a]
        out[..., j, i] = v[..., a] / _MANDEL_W[a]
    return out


def mandel_matrix(C4: np.ndarray) -> np.ndarray:
    M = np.zeros((6, 6))
    for a, (i, j) in enumerate(_MANDEL_IDX):
        for b, (k, l) in enumerate(_MANDEL_IDX):
            M[a, b] = C4[i, j, k, l] * _MANDEL_W[a] * _MANDEL_W[b]
    return M


def reference_medium(mat: Material):
    """Isotropic C0 (the paper gives none; chosen as): 3 k0 = 2 mu0 = (lambda_min + lambda_max) / 2 of the
    crystal's Mandel eigenvalues.  Returns (lam0, mu0)."""
    ev = np.linalg.eigvalsh(mandel_matrix(stiffness_tensor(mat)))
    two_mu = 0.5 * (ev[0] + ev[-1])
    mu0 = 0.5 * two_mu
    k0 = two_mu / 3.0
    lam0 = k0 - 2.0 * mu0 / 3.0
    return lam0, mu0


def bunge_rotation(euler: np.ndarray) -> np.ndarray:
    """Crystal-to-sample rotation R = Rz(phi1) Rx(Phi) Rz(phi2) (Bunge ZXZ, crystal to sample).

    euler (..., 3) rad -> (..., 3, 3); v_sample = R v_crystal.
    Parity: pinned (tests check R e_z and orthogonality against hand values).
    """
    e = np.asarray(euler, dtype=np.float64)
    c1, s1 = np.cos(e[..., 0]), np.sin(e[..., 0])
    c, s = np.cos(e[..., 1]), np.sin(e[..., 1])
    c2, s2 = np.cos(e[..., 2]), np.sin(e[..., 2])
    Rz1 = np.zeros(e.shape[:-1] + (3, 3))
    Rz1[..., 0, 0], Rz1[..., 0, 1], Rz1[..., 1, 0], Rz1[..., 1, 1], Rz1[..., 2, 2] = c1, -s1, s1, c1, 1.0
    Rx = np.zeros(e.shape[:-1] + (3, 3))
    Rx[..., 0, 0], Rx[..., 1, 1], Rx[..., 1, 2], Rx[..., 2, 1], Rx[..., 2, 2] = 1.0, c, -s, s, c
    Rz2 = np.zeros(e.shape[:-1] + (3, 3))
    Rz2[..., 0, 0], Rz2[..., 0, 1], Rz2[..., 1, 0], Rz2[..., 1, 1], Rz2[..., 2, 2] = c2, -s2, s2, c2, 1.0
    return Rz1 @ Rx @ Rz2


# ----------------------------------------------------------------------------------
# Constitutive law (Sec. 3 and Sec. 4)
# ----------------------------------------------------------------------------------
def interaction_matrix(size: int, h_diag: float, h_off: float) -> np.ndarray:
    q = np.full((size, size), h_off)
    np.fill_diagonal(q, h_diag)
    return q


def regularized_rate(a, P, Kn, n, eta):
    """Non-negative rate rho solving rho = P < (a - eta rho) / Kn >^n  (Sec. 4, Eq. (regu)).

    With z = (a - eta rho)/Kn the equation becomes phi(z) = eta P z^n + Kn z - a = 0;
    phi is convex and increasing on z > 0, so Newton from the upper bound
    z0 = min(a/Kn, (a/(eta P))^(1/n)) decreases monotonically to the unique root.
    rho = 0 where a <= 0 or P <= 0.  Iterates until no element moves.
    Parity: pinned (bisection to 1e-15, eta -> 0 and large-a limits).
    """
    a = np.asarray(a, dtype=np.float64)
    P = np.broadcast_to(np.asarray(P, dtype=np.float64), a.shape)
    active = (a > 0.0) & (P > 0.0)
    rho = np.zeros_like(a)
    if not np.any(active):
        return rho
    aa = a[active]
    pp = P[active]
    z = aa / Kn
    if eta > 0.0:
        z = np.minimum(z, (aa / (eta * pp)) ** (1.0 / n))
    for _ in range(200):
        phi = eta * pp * z**n + Kn * z - aa
        dphi = n * eta * pp * z ** (n - 1.0) + Kn
        z_new = np.maximum(z - phi / dphi, 0.0)
        if np.all(z_new >= z):
            break
        z = np.minimum(z, z_new)
    rho[active] = pp * z**n
    return rho


class Constitutive:
    """Crystal-frame Meric-Cailletaud right-hand side, vectorised over voxels."""

    def __init__(self, mat: Material):
        self.mat = mat
        self.C = stiffness_tensor(mat)
        self.m = schmid_tensors()
        self.r0 = mat.r0_vector()
        self.q_slip = interaction_matrix(N_SLIP, mat.h_diag, mat.h_off)
        self.q_twin = interaction_matrix(N_TWIN, mat.h_diag, mat.h_off)

    def stress(self, eps_c, ep):
        """sigma = C : (eps - eps_p) in the crystal frame (Sec. 3, Hooke's law)."""
        return np.einsum("ijkl,vkl->vij", self.C, eps_c - ep)

    def yield_stress(self, v):
        """Isotropic hardening (Sec. 3): r^s = tau0^s + Q_s sum_s' q_ss' (1 - exp(-b_s v^s')),
        slip and twin blocks separately.  v: (V, 16) -> r: (V, 16)."""
        mt = self.mat
        g_slip = 1.0 - np.exp(-mt.b_s * v[:, :N_SLIP])
        g_twin = 1.0 - np.exp(-mt.b_b * v[:, N_SLIP:])
        r_slip = self.r0[:N_SLIP] + mt.Q_s * g_slip @ self.q_slip.T
        r_twin = self.r0[N_SLIP:] + mt.Q_b * g_twin @ self.q_twin.T
        return np.concatenate([r_slip, r_twin], axis=1)

    def rhs(self, eps_c, ep, v, alpha):
        """Rates (ep_dot, v_dot, alpha_dot) at strain eps_c and state (ep, v, alpha).

        eps_c, ep: (V, 3, 3); v: (V, 16) accumulated slip, twin entries are v^beta;
        alpha: (V, 12) kinematic variables of the slip systems (back-stress x = c alpha, not in the paper's text;
        none on the twins).
        """
        mt = self.mat
        sigma = self.stress(eps_c, ep)
        tau = np.einsum("vij,sij->vs", sigma, self.m)
        r = self.yield_stress(v)
        r_slip, r_twin = r[:, :N_SLIP], r[:, N_SLIP:]
        # slip: Norton flow with back-stress x = c alpha, regularised (Sec. 4)
        tau_eff = tau[:, :N_SLIP] - mt.c * alpha
        a_slip = np.abs(tau_eff) - r_slip
        gdot_slip = np.sign(tau_eff) * regularized_rate(a_slip, 1.0, mt.K, mt.n, mt.eta)
        # twinning: unidirectional, f = sqrt(2) v^beta, gamma_dot = f_dot / sqrt(2)
        f_total = SQRT2 * np.sum(v[:, N_SLIP:], axis=1)
        P_twin = (mt.Kc / SQRT2) * np.maximum(0.0, mt.fm - f_total)
        a_twin = tau[:, N_SLIP:] - r_twin
        gdot_twin = regularized_rate(a_twin, P_twin[:, None], mt.Kt, mt.nt, mt.eta)
        # plastic strain rate (Sec. 3), twin-fraction weighting (1 - sum f) on the slip part only
        ep_dot = (1.0 - f_total)[:, None, None] * np.einsum("vs,sij->vij", gdot_slip, self.m[:N_SLIP])
        ep_dot = ep_dot + np.einsum("vb,bij->vij", gdot_twin, self.m[N_SLIP:])
        v_dot = np.concatenate([np.abs(gdot_slip), gdot_twin], axis=1)
        alpha_dot = gdot_slip - mt.d * np.abs(gdot_slip) * alpha
        return ep_dot, v_dot, alpha_dot

    def integrate(self, eps_n_c, eps_c, ep, v, alpha, dt, n_sub):
        """N_sub classical RK4 steps over one increment along the linear strain path
        eps(s) = eps_n + s (eps - eps_n), s in [0, 1] (Sec. 3 end; the paper does not say how the strain varies inside an increment).

        Returns (sigma_c, ep, v, alpha) at the end of the increment.
        Parity: pinned (Radau reference, homogeneous and single-crystal tests).
        """
        h = dt / n_sub
        d_eps = eps_c - eps_n_c
        y = (ep, v, alpha)

        def strain(s):
            return eps_n_c + s * d_eps

        def add(y0, k, w):
            return tuple(a + w * b for a, b in zip(y0, k))

        for m in range(n_sub):
            s0 = m / n_sub
            s_half = (m + 0.5) / n_sub
            s1 = (m + 1.0) / n_sub
            k1 = self.rhs(strain(s0), *y)
            k2 = self.rhs(strain(s_half), *add(y, k1, 0.5 * h))
            k3 = self.rhs(strain(s_half), *add(y, k2, 0.5 * h))
            k4 = self.rhs(strain(s1), *add(y, k3, h))
            y = tuple(
                y0 + (h / 6.0) * (a + 2.0 * b + 2.0 * c + d)
                for y0, a, b, c, d in zip(y, k1, k2, k3, k4)
            )
        ep, v, alpha = y
        return self.stress(eps_c, ep), ep, v, alpha


def von_mises(sig: np.ndarray) -> np.ndarray:
    """sqrt(3/2 s:s) with s the deviator (Sec. 5, equivalent stress).

    Parity: pinned (tests/test_oracle_effective.py: uniaxial stress s gives |s|, pure
    shear t gives sqrt(3) |t|, hydrostatic stress gives 0, rotation invariance).
    """
    s = sig - np.trace(sig, axis1=-2, axis2=-1)[..., None, None] * np.eye(3) / 3.0
    return np.sqrt(1.5 * np.sum(s * s, axis=(-2, -1)))


def effective_averages(v: np.ndarray):
    """The Sec. 5 averages of the internal variables over the RVE: (<f_beta>, <v^s>).

    v: (V, 16) accumulated slip of the 12 slip systems followed by the 4 twin systems.
    <f_beta> is the mean over the 4 twin systems and all voxels of the twin volume
    fraction f = sqrt(2) v^beta (Sec. 3); <v^s> the mean over the 12 slip systems and all
    voxels of v^s (twins excluded).
    Parity: pinned (tests/test_oracle_effective.py: hand-set v on a few voxels).
    """
    mean_f = float(np.mean(SQRT2 * v[:, N_SLIP:]))
    mean_v = float(np.mean(v[:, :N_SLIP]))
    return mean_f, mean_v


# ----------------------------------------------------------------------------------
# Green operator (Willot's rotated discrete scheme)
# ----------------------------------------------------------------------------------
def wave_vectors(shape, scheme: str = "willot"):
    """kappa(xi) on the half spectrum of numpy's rfftn over axes (z, y, x).

    shape = (nz, ny, nx).  Returns an array (nz, ny, nx//2+1, 3) holding (k_x, k_y, k_z).
    "willot": rotated scheme, k_j = sin(q_j/2) prod_{m != j} cos(q_m/2), q_j = 2 pi xi_j / N_j.
    "ms":     continuous frequencies xi_j in (-N/2, N/2), component set to 0 at Nyquist.
    """
    nz, ny, nx = shape
    iz = np.arange(nz)[:, None, None]
    iy = np.arange(ny)[None, :, None]
    ix = np.arange(nx // 2 + 1)[None, None, :]
    out = np.zeros((nz, ny, nx // 2 + 1, 3))
    if scheme == "willot":
        def sc(i, n):  # sin and cos of pi i / n, exact at Nyquist (cos(pi/2) = 0)
            h = np.pi * i / n
            nyq = 2 * i == n
            return np.where(nyq, 1.0, np.sin(h)), np.where(nyq, 0.0, np.cos(h))

        (sx, cx), (sy, cy), (sz, cz) = sc(ix, nx), sc(iy, ny), sc(iz, nz)
        out[..., 0] = sx * cy * cz
        out[..., 1] = cx * sy * cz
        out[..., 2] = cx * cy * sz
    elif scheme == "ms":
        def signed(i, n):
            f = np.where(i <= n // 2, i, i - n).astype(np.float64)
            if n % 2 == 0:
                f = np.where(i == n // 2, 0.0, f)
            return 2.0 * np.pi * f / n

        out[..., 0] = signed(ix, nx) + 0.0 * iy + 0.0 * iz
        out[..., 1] = signed(iy, ny) + 0.0 * ix + 0.0 * iz
        out[..., 2] = signed(iz, nz) + 0.0 * ix + 0.0 * iy
    else:
        raise ValueError(scheme)
    return out


def hermitian_weights(nx: int) -> np.ndarray:
    """Multiplicity of each stored kx of the half spectrum of a real field: 1 for kx = 0
    and (nx even) for the Nyquist plane kx = nx/2, whose conjugate partners are stored
    themselves, 2 for every other kx, which also stands for its unstored partner -kx."""
    w = np.full(nx // 2 + 1, 2.0)
    w[0] = 1.0
    if nx % 2 == 0:
        w[-1] = 1.0
    return w


def equilibrium_error(sig_grid: np.ndarray, kappa: np.ndarray) -> float:
    """Equilibrium error of a stress field (the fixed point's stopping test; the paper
    gives no criterion, so the Moulinec-Suquet measure with the scheme's own wave vectors):

        e = sqrt( sum over all frequencies xi of |kappa(xi) . sigma_hat(xi)|^2 ) / |sigma_hat(0)|

    with the unnormalised transform sigma_hat, the Frobenius norm of the 3x3 tensor
    sigma_hat(0) = N <sigma>, and the sum over the full spectrum taken on the half
    spectrum with hermitian_weights.  sig_grid: (nz, ny, nx, 3, 3) real; kappa:
    wave_vectors(shape).
    Parity: pinned (tests/test_oracle_effective.py: single Fourier modes on the kx = 0
    plane, an interior plane and the Nyquist plane against hand values; divergence-free
    fields give 0).
    """
    nx = sig_grid.shape[2]
    sig_hat = np.fft.rfftn(sig_grid, axes=(0, 1, 2))
    div = np.einsum("zyxij,zyxj->zyxi", sig_hat, kappa)
    num = np.sum(hermitian_weights(nx)[None, None, :] * np.sum(np.abs(div) ** 2, axis=-1))
    denom = np.linalg.norm(sig_hat[0, 0, 0])
    return math.sqrt(num) / denom if denom > 0 else 0.0


def green_tensor(kappa, lam0, mu0):
    """Explicit Gamma0_ijkl(kappa) of an isotropic medium, zero where kappa = 0.

    Gamma_ijkl = (d_ki k_l k_j + d_li k_k k_j + d_kj k_l k_i + d_lj k_k k_i)/(4 mu0 |k|^2)
                 - (lam0 + mu0)/(mu0 (lam0 + 2 mu0)) k_i k_j k_k k_l / |k|^4.
    """
    k = np.asarray(kappa, dtype=np.float64)
    k2 = np.sum(k * k, axis=-1)
    safe = np.where(k2 > 0.0, k2, 1.0)
    d = np.eye(3)
    t1 = (
        np.einsum("ki,...l,...j->...ijkl", d, k, k)
        + np.einsum("li,...k,...j->...ijkl", d, k, k)
        + np.einsum("kj,...l,...i->...ijkl", d, k, k)
        + np.einsum("lj,...k,...i->...ijkl", d, k, k)
    ) / (4.0 * mu0 * safe[..., None, None, None, None])
    t2 = np.einsum("...i,...j,...k,...l->...ijkl", k, k, k, k) / (safe**2)[..., None, None, None, None]
    G = t1 - (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0)) * t2
    return np.where((k2 > 0.0)[..., None, None, None, None], G, 0.0)


def apply_green(kappa, tau_hat, lam0, mu0):
    """eps_hat = -Gamma0(kappa) : tau_hat, written with the contraction of `green_tensor`
    on a symmetric tau (kappa = 0 gives 0).  kappa (..., 3) real, tau_hat (..., 3, 3)."""
    k = kappa
    k2 = np.sum(k * k, axis=-1)
    safe = np.where(k2 > 0.0, k2, 1.0)
    tk = np.einsum("...ij,...j->...i", tau_hat, k)
    ktk = np.einsum("...i,...i->...", k, tk)
    coef = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0))
    sym = k[..., :, None] * tk[..., None, :] + tk[..., :, None] * k[..., None, :]
    g = sym / (2.0 * mu0 * safe[..., None, None]) - coef * k[..., :, None] * k[..., None, :] * (
        ktk / safe**2
    )[..., None, None]
    return -np.where((k2 > 0.0)[..., None, None], g, 0.0)


# ----------------------------------------------------------------------------------
# Full-field solver
# ----------------------------------------------------------------------------------
@dataclass
class Load:
    """Mixed macroscopic load: strain rate on controlled components,
    target mean stress on the others.  Component order (11, 22, 33, 23, 13, 12),
    tensor (not engineering) shear."""

    Edot: np.ndarray = field(default_factory=lambda: np.array([0, 0, 1e-3, 0, 0, 0], dtype=np.float64))
    strain_ctrl: np.ndarray = field(default_factory=lambda: np.array([0, 0, 1, 0, 0, 0], dtype=bool))
    Sigma: np.ndarray = field(default_factory=lambda: np.zeros(6))
    dt: float = 1.0


def default_n_sub(dt: float) -> int:
    """Substeps per increment (the paper gives no rule): the smallest power of two with
    dt/n_sub <= 1/8 s."""
    n = 1
    while dt / n > 0.125 * (1.0 + 1e-12):
        n *= 2
    return n


@dataclass
class Options:
    n_sub: int = 0                # 0: default_n_sub(dt)
    tol: float = 1e-6
    max_iter: int = 500
    fixed_iters: int = 0          # > 0: exactly this many iterations per increment
    scheme: str = "willot"
    c0: tuple | None = None       # (lam0, mu0) of the reference medium; None: reference_medium


def _voigt6_to_tensor(v6):
    t = np.zeros((3, 3))
    for a, (i, j) in enumerate(_MANDEL_IDX):
        t[i, j] = t[j, i] = v6[a]
    return t


def _tensor_to_voigt6(t):
    return np.array([t[i, j] for i, j in _MANDEL_IDX])


class NotConverged(RuntimeError):
    pass


class OracleRVE:
    """Periodic voxel RVE solved by the basic Green-operator fixed point (Sec. 3 end).

    grain_id: (nz, ny, nx) integer map, x fastest in memory; euler: (n_grains, 3) Bunge.
    """

    def __init__(self, grain_id, euler, mat: Material | None = None, opts: Options | None = None):
        self.gid = np.asarray(grain_id).astype(np.int64)
        if self.gid.ndim != 3:
            raise ValueError("grain_id must be (nz, ny, nx)")
        self.shape = self.gid.shape
        self.N = int(self.gid.size)
        self.mat = mat or Material()
        self.opts = opts or Options()
        self.law = Constitutive(self.mat)
        self.R = bunge_rotation(np.asarray(euler, dtype=np.float64))[self.gid.reshape(-1)]   # (V,3,3)
        self.lam0, self.mu0 = self.opts.c0 if self.opts.c0 is not None else reference_medium(self.mat)
        self.C0 = isotropic_tensor(self.lam0, self.mu0)
        self.kappa = wave_vectors(self.shape, self.opts.scheme)
        V = self.N
        # committed state at t_n (sample-frame strain, crystal-frame internal variables)
        self.eps_n = np.zeros((V, 3, 3))
        self.ep = np.zeros((V, 3, 3))
        self.v = np.zeros((V, N_SYS))
        self.alpha = np.zeros((V, N_SLIP))
        self.sigma_n = np.zeros((V, 3, 3))
        self.E = np.zeros(6)          # macroscopic strain E_n
        self.E_prev = np.zeros(6)     # E_{n-1}
        self.time = 0.0
        self.increment = 0
        self.load = Load()
        self.history = []

    # ---- helpers --------------------------------------------------------------
    def set_load(self, load: Load):
        self.load = load

    def _c0_mandel(self):
        return mandel_matrix(self.C0)

    def _to_crystal(self, eps):
        return np.einsum("vki,vkl,vlj->vij", self.R, eps, self.R)

    def _to_sample(self, sig_c):
        return np.einsum("vik,vkl,vjl->vij", self.R, sig_c, self.R)

    def constitutive(self, eps):
        """sigma(x) and the end-of-increment state for the trial strain eps (V, 3, 3)."""
        sig_c, ep, v, alpha = self.law.integrate(
            self._to_crystal(self.eps_n), self._to_crystal(eps), self.ep, self.v, self.alpha,
            self.load.dt, self.opts.n_sub if self.opts.n_sub > 0 else default_n_sub(self.load.dt),
        )
        return self._to_sample(sig_c), ep, v, alpha

    def _grid(self, a):
        return a.reshape(self.shape + (3, 3))

    def _fft(self, t):
        return np.fft.rfftn(self._grid(t), axes=(0, 1, 2))

    def _ifft(self, th):
        return np.fft.irfftn(th, s=self.shape, axes=(0, 1, 2)).reshape(self.N, 3, 3)

    # ---- one increment ----------------------------------------------------------
    def step(self):
        """Advance one increment n -> n+1.  Returns the history record."""
        ld, op = self.load, self.opts
        ctrl = np.asarray(ld.strain_ctrl, dtype=bool)
        free = ~ctrl
        M0 = self._c0_mandel()
        Mff = M0[np.ix_(free, free)]
        # macroscopic strain on controlled components and the initial guess (first increment:
        # free components from C0; later: the previous increment's step)
        dE0 = np.zeros(6)
        if self.increment == 0:
            dE0[ctrl] = np.asarray(ld.Edot, dtype=np.float64)[ctrl] * ld.dt
            if np.any(free):
                dm = dE0 * _MANDEL_W
                dm[free] = -np.linalg.solve(Mff, M0[np.ix_(free, ctrl)] @ dm[ctrl])
                dE0 = dm / _MANDEL_W
        else:
            dE0 = self.E - self.E_prev
            dE0[ctrl] = np.asarray(ld.Edot, dtype=np.float64)[ctrl] * ld.dt
        E = self.E + dE0
        eps = self.eps_n + _voigt6_to_tensor(dE0)[None]
        Sigma_m = np.asarray(ld.Sigma, dtype=np.float64) * _MANDEL_W
        N = float(self.N)
        residuals = []
        it = 0
        while True:
            # local constitutive update and polarisation
            sig, ep_new, v_new, a_new = self.constitutive(eps)
            sig_mean = sig.mean(axis=0)
            tau = sig - np.einsum("ijkl,vkl->vij", self.C0, eps)
            # forward transform of tau; equilibrium and stress-constraint errors
            tau_hat = self._fft(tau)
            e_eq = equilibrium_error(self._grid(sig), self.kappa)
            sm = to_mandel(sig_mean)
            miss = (sm - Sigma_m)[free]
            c_F = float(np.linalg.norm(miss) / np.linalg.norm(sm)) if np.any(free) else 0.0
            residuals.append((e_eq, c_F))
            done = (it + 1 >= op.fixed_iters) if op.fixed_iters > 0 else (e_eq < op.tol and c_F < op.tol)
            if done:
                break
            if it + 1 >= op.max_iter:
                raise NotConverged(f"increment {self.increment + 1}: {op.max_iter} iterations, e={e_eq:.3e}")
            # mixed-load update of the free macroscopic components
            if np.any(free):
                Em = E * _MANDEL_W
                Em[free] -= np.linalg.solve(Mff, miss)
                E = Em / _MANDEL_W
            # Green operator, prescribed mean, inverse transform
            eps_hat = apply_green(self.kappa, tau_hat, self.lam0, self.mu0)
            eps_hat[0, 0, 0] = _voigt6_to_tensor(E) * N
            eps = self._ifft(eps_hat)
            it += 1
        # commit and effective outputs
        self.E_prev = self.E.copy()
        self.E = E
        self.eps_n = eps
        self.ep, self.v, self.alpha = ep_new, v_new, a_new
        self.sigma_n = sig
        self.time += ld.dt
        self.increment += 1
        mean_f, mean_v = effective_averages(self.v)
        rec = {
            "increment": self.increment,
            "time": self.time,
            "E": _tensor_to_voigt6(_voigt6_to_tensor(E)),
            "S": _tensor_to_voigt6(sig_mean),
            "S_eq_of_mean": float(von_mises(sig_mean)),
            "mean_S_eq": float(np.mean(von_mises(sig))),
            "mean_f": mean_f,
            "mean_v": mean_v,
            "iterations": it + 1,
            "residual": residuals[-1][0],
            "stress_residual": residuals[-1][1],
            "residuals": residuals,
        }
        self.history.append(rec)
        return rec

    def run(self, n_increments):
        return [self.step() for _ in range(n_increments)]

    def fields(self):
        """Committed sample-frame fields on the grid: stress, strain, plastic strain
        (crystal frame), v, alpha."""
        return {
            "sigma": self._grid(self.sigma_n),
            "eps": self._grid(self.eps_n),
            "eps_p": self.ep.reshape(self.shape + (3, 3)),
            "v": self.v.reshape(self.shape + (N_SYS,)),
            "alpha": self.alpha.reshape(self.shape + (N_SLIP,)),
        }


# ----------------------------------------------------------------------------------
# Stand-alone steps (for element-wise comparisons)
# ----------------------------------------------------------------------------------
def rfft3(real):
    """Unnormalised forward 3-D real-to-complex transform of (..., nz, ny, nx) fields,
    half spectrum along x (the transform of the Green-operator step)."""
    return np.fft.rfftn(np.asarray(real, dtype=np.float64), axes=(-3, -2, -1))


def material_point_increment(mat: Material, R, eps_n, eps, ep, v, alpha, dt, n_sub):
    """Sample-frame wrapper of Constitutive.integrate for V voxels.

    R (V,3,3) crystal->sample; eps_n, eps (V,3,3) sample frame; ep (V,3,3) crystal frame.
    Returns (sigma (V,3,3) sample frame, ep, v, alpha) at the end of the increment.
    """
    law = Constitutive(mat)
    to_c = lambda t: np.einsum("vki,vkl,vlj->vij", R, t, R)  # noqa: E731
    sig_c, ep1, v1, a1 = law.integrate(to_c(eps_n), to_c(eps), ep, v, alpha, dt, n_sub)
    return np.einsum("vik,vkl,vjl->vij", R, sig_c, R), ep1, v1, a1
