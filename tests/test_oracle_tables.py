"""Pins of the oracle's crystallography and elasticity against values fixed by the paper
(Table 1, Sec. 3 moduli) and by closed forms."""
import math

import numpy as np
import pytest

from oracle import rve_oracle as orc


def test_systems_orthogonal_unit_and_distinct():
    n, l, kinds = orc.system_vectors()
    assert np.allclose(np.sum(n * l, axis=1), 0.0, atol=1e-15)
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0)
    assert np.allclose(np.linalg.norm(l, axis=1), 1.0)
    assert kinds.count("o") == 4 and kinds.count("s") == 8 and kinds.count("t") == 4
    pairs = {(tuple(np.round(a, 12)), tuple(np.round(np.abs(b), 12))) for a, b in zip(n, l)}
    assert len(pairs) == 16  # system 9 read as (1 -1 1)[1 1 0], not the printed duplicate of system 7
    # ordinary dislocations glide along 1/2<110]: no c component (c/a = 1 frame)
    for k, d in zip(kinds, l):
        if k == "o":
            assert d[2] == 0.0


def test_schmid_tensor_symmetric_traceless():
    m = orc.schmid_tensors()
    assert np.allclose(m, m.transpose(0, 2, 1))
    assert np.allclose(np.trace(m, axis1=1, axis2=2), 0.0, atol=1e-16)
    assert np.allclose(np.sum(m * m, axis=(1, 2)), 0.5)  # |m|^2 = 1/2 for unit n orthogonal to l


def test_schmid_factors_along_c_axis():
    """Uniaxial stress along crystal [001]: super systems +-1/sqrt(6), ordinary 0,
    twins -sqrt(2)/3 (tension cannot twin, compression activates all four equally)."""
    m = orc.schmid_tensors()
    _, _, kinds = orc.system_vectors()
    f = m[:, 2, 2]
    for k, v in zip(kinds, f):
        if k == "s":
            assert abs(abs(v) - 1 / math.sqrt(6)) < 1e-15
        elif k == "o":
            assert v == 0.0
        else:
            assert abs(v + math.sqrt(2) / 3) < 1e-15
    assert abs(-math.sqrt(2) / 3 - (-0.4714)) < 1e-4


def test_schmid_factors_along_a_axis():
    m = orc.schmid_tensors()
    # hand values: s1 (11-1)[011] -> 0; s2 (11-1)[101] -> 1/sqrt6; twin 1 (11-1)[112] -> 1/sqrt18
    assert abs(m[0, 0, 0]) < 1e-16
    assert abs(m[1, 0, 0] - 1 / math.sqrt(6)) < 1e-15
    assert abs(m[12, 0, 0] - 1 / math.sqrt(18)) < 1e-15


def test_uniaxial_moduli_closed_form():
    """1/S33 = C33 - 2 C13^2/(C11 + C12) and 1/S11 for the tetragonal moduli of Sec. 3
    with C33 = 178 GPa: 135385.2 MPa along c, 139956.7 MPa along a."""
    mat = orc.Material()
    S = np.linalg.inv(orc.mandel_matrix(orc.stiffness_tensor(mat)))
    assert abs(1 / S[2, 2] - 135385.2) < 0.1
    assert abs(1 / S[0, 0] - 139956.7) < 0.1
    # shear: sigma_23 = 2 C44 eps_23, sigma_12 = 2 C66 eps_12
    C = orc.stiffness_tensor(mat)
    assert C[1, 2, 1, 2] == mat.C44 and C[0, 1, 1, 0] == mat.C66 and C[0, 0, 2, 2] == mat.C13


def test_reference_medium():
    """Mandel eigenvalues {105641.8, 109000, 156000, 210000, 210000, 329358.2} MPa give
    2 mu0 = 3 k0 = 217500 MPa, so mu0 = 108750 and lam0 = 0 (the isotropic reference medium)."""
    ev = np.linalg.eigvalsh(orc.mandel_matrix(orc.stiffness_tensor(orc.Material())))
    assert np.allclose(ev, [105641.8, 109000, 156000, 210000, 210000, 329358.2], atol=0.1)
    lam0, mu0 = orc.reference_medium(orc.Material())
    assert abs(mu0 - 108750.0) < 1e-8 and abs(lam0) < 1e-8


def test_bunge_rotation_against_scipy():
    pytest.importorskip("scipy")
    from scipy.spatial.transform import Rotation

    rng = np.random.default_rng(0)
    e = rng.uniform(0, 2 * np.pi, size=(20, 3))
    e[:, 1] = rng.uniform(0, np.pi, size=20)
    R = orc.bunge_rotation(e)
    ref = Rotation.from_euler("ZXZ", e).as_matrix()  # intrinsic z-x'-z''
    assert np.allclose(R, ref, atol=1e-14)
    # hand value: Phi alone tilts the crystal c axis to (0, -sin Phi, cos Phi)
    Rp = orc.bunge_rotation(np.array([0.0, 0.3, 0.0]))
    assert np.allclose(Rp @ [0, 0, 1], [0, -math.sin(0.3), math.cos(0.3)])


def test_mandel_roundtrip_is_isometry():
    rng = np.random.default_rng(1)
    t = rng.normal(size=(5, 3, 3))
    t = t + t.transpose(0, 2, 1)
    v = orc.to_mandel(t)
    assert np.allclose(orc.from_mandel(v), t)
    assert np.allclose(np.sum(v * v, axis=1), np.sum(t * t, axis=(1, 2)))
