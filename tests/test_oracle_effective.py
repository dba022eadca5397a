"""Pins of the oracle's Sec. 5 effective measures and of its equilibrium error against
closed forms: the von Mises stress of textbook stress states, the <f_beta> / <v^s>
averages on hand-set internal variables, and the equilibrium error of single Fourier
modes (each plane class of the half spectrum) and of divergence-free fields."""
import math

import numpy as np
import pytest

from oracle import rve_oracle as orc


def _sym(i, j):
    e = np.zeros((3, 3))
    e[i, j] = e[j, i] = 1.0
    return e


# ---- von Mises equivalent stress (Sec. 5) ---------------------------------------------
def test_von_mises_uniaxial_stress_is_its_magnitude():
    for axis in range(3):
        for s in (250.0, -80.0):
            assert abs(orc.von_mises(s * _sym(axis, axis)) - abs(s)) < 1e-12 * abs(s)


def test_von_mises_pure_shear_is_sqrt3_times_shear():
    t = 40.0
    for i, j in ((0, 1), (1, 2), (0, 2)):
        assert abs(orc.von_mises(t * _sym(i, j)) - math.sqrt(3.0) * t) < 1e-12 * t
    # the same state in principal axes: diag(t, -t, 0)
    assert abs(orc.von_mises(np.diag([t, -t, 0.0])) - math.sqrt(3.0) * t) < 1e-12 * t


def test_von_mises_ignores_hydrostatic_stress():
    assert orc.von_mises(-130.0 * np.eye(3)) < 1e-12
    # equibiaxial tension s = uniaxial compression -s plus a hydrostatic s
    assert abs(orc.von_mises(np.diag([70.0, 70.0, 0.0])) - 70.0) < 1e-12 * 70.0
    assert abs(orc.von_mises(250.0 * _sym(2, 2) + 55.0 * np.eye(3)) - 250.0) < 1e-12 * 250.0


def test_von_mises_is_rotation_invariant_and_vectorised():
    rng = np.random.default_rng(4)
    a = rng.normal(size=(5, 3, 3)) * 100.0
    sig = a + np.swapaxes(a, -1, -2)
    R = orc.bunge_rotation(rng.uniform(0, 3, size=(5, 3)))
    rot = np.einsum("vik,vkl,vjl->vij", R, sig, R)
    got = orc.von_mises(sig)
    assert got.shape == (5,)
    assert np.allclose(orc.von_mises(rot), got, rtol=1e-13)
    # principal-stress form sqrt(((s1-s2)^2 + (s2-s3)^2 + (s3-s1)^2) / 2)
    for v in range(5):
        p = np.linalg.eigvalsh(sig[v])
        ref = math.sqrt(0.5 * ((p[0] - p[1]) ** 2 + (p[1] - p[2]) ** 2 + (p[2] - p[0]) ** 2))
        assert abs(got[v] - ref) < 1e-12 * ref


# ---- <f_beta> and <v^s> (Sec. 5 averages; f = sqrt(2) v, Sec. 3) -------------------------
def test_effective_averages_hand_values():
    v = np.zeros((3, 16))
    v[0, :12] = 0.3
    v[1, :12] = 0.01 * np.arange(12)
    v[0, 12:] = [0.01, 0.0, 0.0, 0.03]
    v[1, 12:] = [0.0, 0.02, 0.0, 0.0]
    v[2, 12:] = [0.0, 0.0, 0.0, 0.04]
    mean_f, mean_v = orc.effective_averages(v)
    # <v^s>: (12 * 0.3 + 0.01 * 66 + 0) / (3 voxels * 12 slip systems)
    assert abs(mean_v - 4.26 / 36.0) < 1e-15
    # <f_beta>: sqrt(2) * (0.01 + 0.03 + 0.02 + 0.04) / (3 voxels * 4 twin systems)
    assert abs(mean_f - math.sqrt(2.0) * 0.10 / 12.0) < 1e-15


def test_effective_averages_separate_slip_from_twins():
    v = np.zeros((2, 16))
    v[:, 12:] = 0.5  # twins only: no slip average
    mean_f, mean_v = orc.effective_averages(v)
    assert mean_v == 0.0 and abs(mean_f - math.sqrt(2.0) * 0.5) < 1e-15
    v = np.zeros((2, 16))
    v[:, :12] = 0.25  # slip only: no twin fraction
    mean_f, mean_v = orc.effective_averages(v)
    assert mean_f == 0.0 and abs(mean_v - 0.25) < 1e-15


def test_increment_record_uses_the_pinned_measures():
    rng = np.random.default_rng(2)
    gid = rng.integers(0, 2, size=(4, 4, 6))
    rve = orc.OracleRVE(gid, np.array([[0.3, 0.9, 1.7], [2.1, 1.2, 0.4]]), opts=orc.Options(fixed_iters=4))
    rve.set_load(orc.Load(dt=1.0))
    for _ in range(3):
        rec = rve.step()
    mean = rve.sigma_n.mean(axis=0)
    assert rec["S_eq_of_mean"] == float(orc.von_mises(mean))
    assert rec["mean_S_eq"] == float(np.mean(orc.von_mises(rve.sigma_n)))
    assert (rec["mean_f"], rec["mean_v"]) == orc.effective_averages(rve.v)
    assert rec["mean_v"] > 0.0
    assert rec["residual"] == orc.equilibrium_error(rve._grid(rve.sigma_n), rve.kappa)


# ---- equilibrium error -------------------------------------------------------------------
SHAPE = (4, 6, 8)  # (nz, ny, nx)
S0 = 100.0 * _sym(2, 2) + 10.0 * _sym(0, 2)  # mean stress, |S0|_F = sqrt(100^2 + 2 * 10^2)
S0_NORM = math.sqrt(100.0**2 + 2.0 * 10.0**2)


def _mode_field(A, profile):
    """S0 + A * profile(i, j, k) on the (nz, ny, nx) grid."""
    nz, ny, nx = SHAPE
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return S0 + profile(i, j, k)[..., None, None] * A


def test_equilibrium_error_interior_kx_plane():
    """cos(2 pi x / nx): sigma_hat(kx = 1) = N/2 A, stored once with weight 2 for its
    unstored partner; Willot kappa = (sin(pi/nx), 0, 0), so
    e = sin(pi/nx) sqrt((A_xx^2 + A_yx^2) / 2) / |S0|."""
    nx = SHAPE[2]
    A = 3.0 * _sym(0, 0) + 4.0 * _sym(0, 1)
    sig = _mode_field(A, lambda i, j, k: np.cos(2 * np.pi * i / nx))
    ref = math.sin(math.pi / nx) * math.sqrt((3.0**2 + 4.0**2) / 2.0) / S0_NORM
    got = orc.equilibrium_error(sig, orc.wave_vectors(SHAPE))
    assert abs(got - ref) < 1e-13 * ref


def test_equilibrium_error_kx_zero_plane():
    """cos(2 pi y / ny): both ky = 1 and ky = ny - 1 sit on the stored kx = 0 plane (weight
    1 each, N/2 A each); kappa = (0, sin(pi/ny), 0) = (0, 1/2, 0) for ny = 6, so
    e = (1/2) sqrt((A_yy^2 + A_zy^2) / 2) / |S0|."""
    ny = SHAPE[1]
    A = 5.0 * _sym(1, 1) + 2.0 * _sym(1, 2)
    sig = _mode_field(A, lambda i, j, k: np.cos(2 * np.pi * j / ny))
    ref = 0.5 * math.sqrt((5.0**2 + 2.0**2) / 2.0) / S0_NORM
    got = orc.equilibrium_error(sig, orc.wave_vectors(SHAPE))
    assert abs(got - ref) < 1e-13 * ref


def test_equilibrium_error_nyquist_plane():
    """(-1)^i: all of it at kx = nx/2 (sigma_hat = N A, weight 1), where the rotated
    scheme's kappa is (1, 0, 0), so e = |A e_x| / |S0|."""
    A = 6.0 * _sym(0, 0) + 2.0 * _sym(0, 2)
    sig = _mode_field(A, lambda i, j, k: (-1.0) ** i)
    ref = math.sqrt(6.0**2 + 2.0**2) / S0_NORM
    got = orc.equilibrium_error(sig, orc.wave_vectors(SHAPE))
    assert abs(got - ref) < 1e-13 * ref


@pytest.mark.parametrize("scheme", ["willot", "ms"])
def test_equilibrium_error_divergence_free_fields(scheme):
    """sigma_zz varying along x only, and sigma_xy varying along z only, are equilibrated."""
    kap = orc.wave_vectors(SHAPE, scheme)
    nz, _, nx = SHAPE
    sig = _mode_field(40.0 * _sym(2, 2), lambda i, j, k: np.cos(2 * np.pi * i / nx) + 0.5 * np.sin(4 * np.pi * i / nx))
    assert orc.equilibrium_error(sig, kap) < 1e-15
    sig = _mode_field(25.0 * _sym(0, 1), lambda i, j, k: np.sin(2 * np.pi * k / nz))
    assert orc.equilibrium_error(sig, kap) < 1e-15
    assert orc.equilibrium_error(_mode_field(0.0 * S0, lambda i, j, k: i), kap) == 0.0


def test_hermitian_weights():
    assert orc.hermitian_weights(8).tolist() == [1.0, 2.0, 2.0, 2.0, 1.0]
    assert orc.hermitian_weights(2).tolist() == [1.0, 1.0]
    assert orc.hermitian_weights(5).tolist() == [1.0, 2.0, 2.0]
