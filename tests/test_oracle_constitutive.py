"""Pins of the oracle's Meric-Cailletaud law (Sec. 3), its viscous regularisation
(Sec. 4) and its RK4 integration."""
import math

import numpy as np
import pytest

from oracle import rve_oracle as orc


def _bisect_rate(a, P, K, n, eta):
    """rho in [0, hi] with rho - P <(a - eta rho)/K>^n = 0, by plain bisection."""
    f = lambda r: r - P * max(0.0, (a - eta * r) / K) ** n  # noqa: E731
    hi = a / eta if eta > 0 else P * (a / K) ** n
    lo = 0.0
    for _ in range(3000):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if f(mid) > 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("n", [10.0, 6.42])
@pytest.mark.parametrize("eta", [1e4, 1e2, 1.0])
def test_regularized_rate_vs_bisection(n, eta):
    rng = np.random.default_rng(int(n * 100 + eta))
    a = rng.uniform(1e-3, 400.0, size=40)
    P = rng.choice([1.0, 0.37], size=40)
    got = orc.regularized_rate(a, P, 10.0, n, eta)
    for i in range(40):
        ref = _bisect_rate(a[i], P[i], 10.0, n, eta)
        assert abs(got[i] - ref) <= 1e-13 * ref + 1e-300, (a[i], got[i], ref)


def test_regularized_rate_limits():
    # no driving force, or no twin capacity left: no flow
    assert np.all(orc.regularized_rate(np.array([-5.0, 0.0, 3.0]), np.array([1.0, 1.0, 0.0]), 10.0, 10.0, 1e4) == 0.0)
    # eta = 0: plain Norton <a/K>^n
    a = np.array([1.0, 17.0, 55.0])
    assert np.allclose(orc.regularized_rate(a, 1.0, 10.0, 10.0, 0.0), (a / 10.0) ** 10, rtol=1e-14)
    # large overstress: eta rho -> a (the viscous term carries the load)
    r = orc.regularized_rate(np.array([1e7]), 1.0, 10.0, 10.0, 1e4)[0]
    assert abs(1e4 * r / 1e7 - 1) < 1e-5
    # the root satisfies its equation
    r = orc.regularized_rate(np.array([30.0]), 1.0, 10.0, 10.0, 1e4)[0]
    assert abs(r - ((30.0 - 1e4 * r) / 10.0) ** 10) < 1e-15


def test_interaction_matrix_structure():
    """r = r0 + Q sum q (1 - e^{-b v}), q = 1 on, 1.2 off the diagonal within each block."""
    law = orc.Constitutive(orc.Material())
    r = law.yield_stress(np.zeros((1, 16)))[0]
    assert np.allclose(r[:12], [200, 200, 90] * 4) and np.allclose(r[12:], 110)
    v = np.zeros((1, 16))
    v[0, 0] = 1e3  # saturate system 1 only
    r = law.yield_stress(v)[0]
    assert abs(r[0] - 220.0) < 1e-12 and abs(r[1] - 224.0) < 1e-12 and abs(r[2] - 114.0) < 1e-12
    assert np.allclose(r[12:], 110.0)
    r = law.yield_stress(np.full((1, 16), 1e3))[0]
    assert np.allclose(r[:12], np.array([200, 200, 90] * 4) + 20 * (1 + 11 * 1.2))
    assert np.allclose(r[12:], 110 + 20 * (1 + 3 * 1.2))
    # b sets the saturation rate: half-way at v = ln 2 / b
    v = np.zeros((1, 16))
    v[0, 5] = math.log(2) / 5.0
    assert abs(law.yield_stress(v)[0, 5] - (90 + 10.0)) < 1e-12


def _uniaxial_strain(mat, sigma_zz):
    """Crystal-frame strain of a uniaxial stress along [001] (compliance of Sec. 3 moduli)."""
    S = np.linalg.inv(orc.mandel_matrix(orc.stiffness_tensor(mat)))
    return orc.from_mandel(S @ np.array([0, 0, sigma_zz, 0, 0, 0.0]))


def test_twinning_is_unidirectional():
    mat = orc.Material()
    law = orc.Constitutive(mat)
    z = np.zeros((1, 3, 3))
    for sig, expect in ((+600.0, False), (-600.0, True)):
        ep_dot, v_dot, _ = law.rhs(_uniaxial_strain(mat, sig)[None], z, np.zeros((1, 16)), np.zeros((1, 12)))
        tw = v_dot[0, 12:]
        if expect:
            assert np.all(tw > 0) and np.allclose(tw, tw[0], rtol=1e-12)
        else:
            assert np.all(tw == 0)
        # plastic incompressibility
        assert abs(np.trace(ep_dot[0])) < 1e-15 * np.abs(ep_dot).max() + 1e-30
    # no twin capacity left: sum f >= fm stops twinning
    v = np.zeros((1, 16))
    v[0, 12:] = mat.fm / math.sqrt(2) / 4 * 1.01
    _, v_dot, _ = law.rhs(_uniaxial_strain(mat, -600.0)[None], z, v, np.zeros((1, 12)))
    assert np.all(v_dot[0, 12:] == 0)


def test_slip_rate_sign_and_kinematic_law():
    """Pure resolved shear on ordinary system 3 at 1.05 r0 activates that system alone:
    gamma_dot takes the sign of tau - x, v_dot = |gamma_dot|, alpha_dot = gamma_dot -
    d |gamma_dot| alpha, eps_p_dot = gamma_dot m; with twins present the weighting
    (1 - sum f) scales the slip part only (as written in Sec. 3)."""
    mat = orc.Material()
    law = orc.Constitutive(mat)
    k = 2
    mk = law.m[k]
    S = np.linalg.inv(orc.mandel_matrix(law.C))
    for sgn in (+1.0, -1.0):
        sig = sgn * 1.05 * 90.0 * mk / np.sum(mk * mk)
        eps = orc.from_mandel(S @ orc.to_mandel(sig))[None]
        al = np.zeros((1, 12))
        al[0, k] = -sgn * 1e-4  # back-stress x = c alpha = -sgn MPa
        ep_dot, v_dot, al_dot = law.rhs(eps, np.zeros((1, 3, 3)), np.zeros((1, 16)), al)
        active = np.nonzero(v_dot[0])[0]
        assert list(active) == [k]
        g = al_dot[0, k] + mat.d * v_dot[0, k] * al[0, k]
        assert np.sign(g) == sgn and abs(abs(g) - v_dot[0, k]) < 1e-18
        a = abs(sgn * 94.5 + sgn * 1.0) - 90.0
        assert abs(v_dot[0, k] - orc.regularized_rate(np.array([a]), 1.0, mat.K, mat.n, mat.eta)[0]) < 1e-18
        assert np.allclose(ep_dot[0], g * mk, rtol=1e-13, atol=0)
        assert np.allclose(al_dot[0, np.arange(12) != k], 0.0)
    v = np.zeros((1, 16))
    v[0, 12] = 0.1 / math.sqrt(2)  # f_total = 0.1
    sig = 1.05 * 90.0 * mk / np.sum(mk * mk)
    eps = orc.from_mandel(S @ orc.to_mandel(sig))[None]
    ep0, vd0, _ = law.rhs(eps, np.zeros((1, 3, 3)), np.zeros((1, 16)), np.zeros((1, 12)))
    ep1, vd1, _ = law.rhs(eps, np.zeros((1, 3, 3)), v, np.zeros((1, 12)))
    assert vd1[0, k] == vd0[0, k]  # slip rate itself is not weighted
    assert np.allclose(ep1[0], 0.9 * ep0[0], rtol=1e-13, atol=0)


def _radau_reference(mat, R, eps_n, eps, dt):
    from scipy.integrate import solve_ivp

    law = orc.Constitutive(mat)
    e0 = R.T @ eps_n @ R
    e1 = R.T @ eps @ R

    def f(t, y):
        ep = y[:9].reshape(1, 3, 3)
        v = y[9:25][None]
        al = y[25:][None]
        d_ep, d_v, d_al = law.rhs((e0 + (t / dt) * (e1 - e0))[None], ep, v, al)
        return np.concatenate([d_ep.ravel(), d_v.ravel(), d_al.ravel()])

    sol = solve_ivp(f, (0.0, dt), np.zeros(37), method="Radau", rtol=1e-11, atol=1e-16)
    y = sol.y[:, -1]
    return y[:9].reshape(3, 3), y[9:25], y[25:]


def test_rk4_matches_radau():
    pytest.importorskip("scipy")
    mat = orc.Material()
    law = orc.Constitutive(mat)
    R = orc.bunge_rotation(np.array([0.4, 1.1, 2.3]))
    eps_n = np.zeros((3, 3))
    eps = np.diag([-0.8e-3, -0.7e-3, 2.5e-3])
    ep_r, v_r, al_r = _radau_reference(mat, R, eps_n, eps, 1.0)
    to_c = lambda t: (R.T @ t @ R)[None]  # noqa: E731
    _, ep, v, al = law.integrate(to_c(eps_n), to_c(eps), np.zeros((1, 3, 3)), np.zeros((1, 16)), np.zeros((1, 12)), 1.0, 256)
    assert np.abs(v_r).max() > 1e-4  # plastic flow happened
    assert np.abs(ep[0] - ep_r).max() < 1e-8 * np.abs(ep_r).max()
    assert np.abs(v[0] - v_r).max() < 1e-8 * np.abs(v_r).max()
    assert np.abs(al[0] - al_r).max() < 1e-8 * np.abs(al_r).max()


def test_rk4_fourth_order_on_smooth_flow():
    """Zero thresholds (every system flowing, no activation kinks), twins off: halving the
    substep divides the error by ~16."""
    mat = orc.Material(r0_ord=0.0, r0_sup=0.0, Q_s=0.0, Kc=0.0, c=0.0)
    law = orc.Constitutive(mat)
    R = orc.bunge_rotation(np.array([0.2, 0.5, 0.9]))
    e0 = (R.T @ np.diag([4e-4, -2e-4, 1e-3]) @ R)[None]
    e1 = (R.T @ np.diag([6e-4, -1e-4, 2.2e-3]) @ R)[None]
    z = (np.zeros((1, 3, 3)), np.zeros((1, 16)), np.zeros((1, 12)))
    ref = law.integrate(e0, e1, *z, 0.5, 1024)[0]
    errs = [np.abs(law.integrate(e0, e1, *z, 0.5, n)[0] - ref).max() for n in (16, 32, 64)]
    assert 13.0 < errs[0] / errs[1] < 20.0 and 13.0 < errs[1] / errs[2] < 20.0
