"""Pins of the oracle's Green operator and discrete wave vectors (Willot's rotated scheme)."""
import numpy as np

from oracle import rve_oracle as orc


def _random_sym(rng, shape, complex_=False):
    a = rng.normal(size=shape + (3, 3))
    if complex_:
        a = a + 1j * rng.normal(size=shape + (3, 3))
    return 0.5 * (a + np.swapaxes(a, -1, -2))


def _ddot(G, H):
    return np.einsum("ijkl,klmn->ijmn", G, H)


def test_green_symmetries_and_projection():
    rng = np.random.default_rng(2)
    lam0, mu0 = 31.0, 47.0
    C0 = orc.isotropic_tensor(lam0, mu0)
    for _ in range(10):
        k = rng.normal(size=3)
        G = orc.green_tensor(k, lam0, mu0)
        assert np.allclose(G, G.transpose(1, 0, 2, 3))
        assert np.allclose(G, G.transpose(0, 1, 3, 2))
        assert np.allclose(G, G.transpose(2, 3, 0, 1))
        # Gamma : C0 : Gamma = Gamma (projection)
        assert np.allclose(_ddot(_ddot(G, C0), G), G, atol=1e-14)
        # homogeneous of degree 0
        assert np.allclose(orc.green_tensor(3.7 * k, lam0, mu0), G)
    assert np.all(orc.green_tensor(np.zeros(3), lam0, mu0) == 0.0)


def test_green_reproduces_compatible_and_kills_equilibrated():
    rng = np.random.default_rng(3)
    lam0, mu0 = 12.0, 30.0
    C0 = orc.isotropic_tensor(lam0, mu0)
    for _ in range(10):
        k = rng.normal(size=3)
        u = rng.normal(size=3)
        comp = 0.5 * (np.outer(k, u) + np.outer(u, k))
        G = orc.green_tensor(k, lam0, mu0)
        assert np.allclose(np.einsum("ijkl,kl->ij", G, np.einsum("ijkl,kl->ij", C0, comp)), comp)
        # equilibrated: sigma k = 0
        P = np.eye(3) - np.outer(k, k) / (k @ k)
        s = _random_sym(rng, ())
        eq = P @ s @ P
        assert np.allclose(eq @ k, 0.0)
        assert np.allclose(np.einsum("ijkl,kl->ij", G, eq), 0.0, atol=1e-15)


def test_apply_green_equals_acoustic_tensor_solve():
    """eps = -sym(k x u) with A(k) u = tau k and A_ik = C0_ijkl k_j k_l (displacement form)."""
    rng = np.random.default_rng(4)
    lam0, mu0 = 0.0, 108750.0
    d = np.eye(3)
    C0 = lam0 * np.einsum("ij,kl->ijkl", d, d) + mu0 * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d))
    k = rng.normal(size=(50, 3))
    tau = _random_sym(rng, (50,), complex_=True)
    got = orc.apply_green(k, tau, lam0, mu0)
    for a in range(50):
        A = np.einsum("ijkl,j,l->ik", C0, k[a], k[a])
        u = np.linalg.solve(A, tau[a] @ k[a])
        ref = -0.5 * (np.outer(k[a], u) + np.outer(u, k[a]))
        assert np.allclose(got[a], ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
        assert np.allclose(got[a], -np.einsum("ijkl,kl->ij", orc.green_tensor(k[a], lam0, mu0), tau[a]))


def test_willot_wave_vector_is_trilinear_gradient():
    """k_j = (i/4)(e^{i q_j} - 1) prod_{m != j}(1 + e^{i q_m}) equals -2 e^{i sum(q)/2} kappa_j."""
    shape = (6, 10, 8)
    kap = orc.wave_vectors(shape, "willot")
    nz, ny, nx = shape
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx // 2 + 1), indexing="ij")
    q = [2 * np.pi * ix / nx, 2 * np.pi * iy / ny, 2 * np.pi * iz / nz]
    e = [np.exp(1j * qq) for qq in q]
    kd = np.stack([
        0.25j * (e[0] - 1) * (1 + e[1]) * (1 + e[2]),
        0.25j * (e[1] - 1) * (1 + e[0]) * (1 + e[2]),
        0.25j * (e[2] - 1) * (1 + e[0]) * (1 + e[1]),
    ], axis=-1)
    phase = -2 * np.exp(0.5j * (q[0] + q[1] + q[2]))
    assert np.allclose(kd, phase[..., None] * kap, atol=1e-14)
    # zero at the origin and where two components are at Nyquist
    assert np.all(kap[0, 0, 0] == 0)
    assert np.all(kap[0, ny // 2, nx // 2] == 0.0) and np.all(kap[2, ny // 2, nx // 2] == 0.0)


def test_ms_wave_vector():
    kap = orc.wave_vectors((4, 6, 8), "ms")
    assert np.allclose(kap[1, 5, 3], [2 * np.pi * 3 / 8, 2 * np.pi * -1 / 6, 2 * np.pi * 1 / 4])
    assert kap[0, 3, 4, 0] == 0 and kap[0, 3, 4, 1] == 0  # Nyquist components zeroed
