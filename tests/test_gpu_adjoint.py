"""Reverse pass of the per-voxel constitutive update (rve_material_point_vjp) against
central finite differences of the FP64 oracle's material-point update (Sec. 3 law, Sec. 4
regularised rates, RK4): directional derivatives of J = sum(sigma_b . sigma) +
sum(state_b . state) with respect to every input and each material parameter."""
import dataclasses

import numpy as np
import pytest

from helpers import six_to_tensor, tensor_to_six
from oracle import rve_oracle as orc

pytestmark = pytest.mark.gpu

PARAMS = ["r0_ord", "r0_sup", "r0_twin", "Q_s", "Q_b", "b_s", "b_b", "c", "d"]
PAPER = dict(C33=183000.0, r0_ord=130.0, r0_sup=200.0, r0_twin=130.0, K=104.0, Kt=104.0, n=6.42, nt=6.42,
             Q_s=9.57, Q_b=10.5, Kc=1.45, fm=0.8, eta=1.0e4, c=5000.0, d=300.0)


def _points(n, seed, scale):
    rng = np.random.default_rng(seed)
    e = rng.uniform(0, 2 * np.pi, size=(n, 3))
    e[:, 1] = np.arccos(rng.uniform(-1, 1, size=n))
    R = orc.bunge_rotation(e)
    sym = lambda a: 0.5 * (a + a.transpose(0, 2, 1))  # noqa: E731
    eps_n = sym(rng.normal(scale=1.5e-3 * scale, size=(n, 3, 3)))
    eps = eps_n + sym(rng.normal(scale=1.0e-3 * scale, size=(n, 3, 3)))
    quiet = rng.uniform(size=n) < 0.25
    eps_n[quiet] *= 0.1
    eps[quiet] *= 0.1
    ep = sym(rng.normal(scale=3e-4, size=(n, 3, 3)))
    ep -= np.trace(ep, axis1=1, axis2=2)[:, None, None] * np.eye(3) / 3
    v = rng.uniform(0, 2e-3, size=(n, 16))
    v[:, 12:] *= 0.1
    al = rng.uniform(-1e-3, 1e-3, size=(n, 12))
    return R, tensor_to_six(eps_n), tensor_to_six(eps), tensor_to_six(ep), v, al


def _J(mat, R, en6, e6, ep6, v, al, sb, yb, dt, nsub):
    sig, ep1, v1, al1 = orc.material_point_increment(mat, R, six_to_tensor(en6), six_to_tensor(e6),
                                                     six_to_tensor(ep6), v, al, dt, nsub)
    y = np.concatenate([tensor_to_six(ep1), v1.T, al1.T], axis=0)
    return float(np.sum(sb * tensor_to_six(sig)) + np.sum(yb * y))


@pytest.mark.parametrize("which", ["workload", "paper"])
def test_material_point_vjp_matches_oracle_finite_differences(lib, cuda, which):
    import torch

    from paper_2402_09996_gb300 import rve

    kw = {} if which == "workload" else PAPER
    mat = dataclasses.replace(orc.Material(), **kw)
    n, dt = 40, 0.5
    nsub = orc.default_n_sub(dt)
    R, en6, e6, ep6, v, al = _points(n, 5 if which == "workload" else 6, 1.0 if which == "workload" else 3.0)
    rng = np.random.default_rng(77)
    sb = rng.normal(size=(6, n)) * 1e-2
    yb = rng.normal(size=(34, n)) * 10.0
    to = lambda a: torch.tensor(np.ascontiguousarray(a), device=cuda, dtype=torch.float64)  # noqa: E731
    state = np.concatenate([ep6, v.T, al.T], axis=0)
    st_b = to(yb)
    eps_b, eps_n_b, R_b, p_b = rve.material_point_vjp(to(R.reshape(n, 9)), to(en6), to(e6), to(state), to(sb), st_b,
                                                      dt, nsub, rve.FP64, **kw)
    eps_b, eps_n_b, R_b, p_b, y0_b = (t.cpu().numpy() for t in (eps_b, eps_n_b, R_b, p_b, st_b))
    J = lambda **ch: _J(ch.get("mat", mat), ch.get("R", R), ch.get("en6", en6), ch.get("e6", e6),  # noqa: E731
                        ch.get("ep6", ep6), ch.get("v", v), ch.get("al", al), sb, yb, dt, nsub)

    def fd(name, base, grad, scale):
        d = np.random.default_rng(sum(map(ord, name))).normal(size=base.shape) * scale
        h = 1e-5
        jp = J(**{name: base + h * d})
        jm = J(**{name: base - h * d})
        num = (jp - jm) / (2 * h)
        ana = float(np.sum(grad * d))
        assert abs(num - ana) <= 2e-6 * max(abs(num), abs(ana)) + 1e-10, (name, num, ana)

    fd("e6", e6, eps_b, 1e-3)
    fd("en6", en6, eps_n_b, 1e-3)
    fd("ep6", ep6, y0_b[:6], 3e-4)
    fd("v", v, y0_b[6:22].T, 1e-3)
    fd("al", al, y0_b[22:].T, 1e-3)
    fd("R", R, R_b.T.reshape(n, 3, 3), 1e-2)
    # parameters: one at a time
    for k, name in enumerate(PARAMS):
        p0 = getattr(mat, name)
        h = 1e-6 * max(abs(p0), 1.0)
        num = (J(mat=dataclasses.replace(mat, **{name: p0 + h})) - J(mat=dataclasses.replace(mat, **{name: p0 - h}))) / (
            2 * h)
        ana = float(np.sum(p_b[k]))
        assert abs(num - ana) <= 2e-5 * max(abs(num), abs(ana)) + 1e-8, (name, num, ana)
    # the sample mixes elastic and plastic points
    _, _, v1, _ = orc.material_point_increment(mat, R, six_to_tensor(en6), six_to_tensor(e6), six_to_tensor(ep6), v,
                                               al, dt, nsub)
    active = np.any(v1 > v, axis=1)
    assert 0.2 < active.mean() < 0.95


def _history_J(gid, euler, mat, target, n_inc, dt, **opts):
    from paper_2402_09996_gb300 import rve

    with rve.RVE(gid, euler, precision=rve.FP64, **opts) as s:
        if mat:
            s.set_material(**mat)
        s.set_mixed_load(dt=dt)
        s.step(n_inc)
        S33 = np.array([h["S"][2] for h in s.history()])
    return float(np.sum((S33 - target) ** 2)), S33


def test_load_history_gradient_matches_finite_differences(lib, cuda):
    """Adjoint of a 4-increment history (checkpoints every 2 increments, replayed) for
    J = sum_n (<sigma_zz>_n - target_n)^2: gradient in the 9 material parameters and the
    Bunge angles of two grains against central differences of the forward solve."""
    from oracle.voronoi import label_rve

    from paper_2402_09996_gb300 import inputs, rve

    inp = inputs.make_inputs((8, 10, 12), 4, 0.0, seed=21)
    gid = label_rve(inp)
    euler = inp.euler[:4].copy()
    n_inc, dt = 4, 0.5
    opts = dict(tol=1e-12, max_iter=3000)
    _, S0 = _history_J(gid, euler, {}, np.zeros(n_inc), n_inc, dt, **opts)
    target = 0.97 * S0
    J, gp, ge, info = rve.history_gradient(gid, euler, n_inc, dt, target, checkpoint_every=2, **opts)
    assert abs(J - float(np.sum((S0 - target) ** 2))) < 1e-9 * J
    assert info["checkpoints"] == [0, 2]
    base = orc.Material()
    for k, name in enumerate(rve.PARAM_NAMES):
        p0 = getattr(base, name)
        h = 1e-5 * abs(p0)
        jp, _ = _history_J(gid, euler, {name: p0 + h}, target, n_inc, dt, **opts)
        jm, _ = _history_J(gid, euler, {name: p0 - h}, target, n_inc, dt, **opts)
        num = (jp - jm) / (2 * h)
        assert abs(num - gp[k]) <= 1e-4 * max(abs(num), abs(gp[k])) + 1e-9 * J / abs(p0), (name, num, gp[k])
    for g in (0, 1):
        for a in range(3):
            h = 1e-5
            ep, em = euler.copy(), euler.copy()
            ep[g, a] += h
            em[g, a] -= h
            num = (_history_J(gid, ep, {}, target, n_inc, dt, **opts)[0] -
                   _history_J(gid, em, {}, target, n_inc, dt, **opts)[0]) / (2 * h)
            assert abs(num - ge[g, a]) <= 1e-4 * max(abs(num), abs(ge[g, a])) + 1e-9 * J, (g, a, num, ge[g, a])


def _history_S33(gid, euler, n_inc, dt, precision):
    from paper_2402_09996_gb300 import rve

    with rve.RVE(gid, euler, precision=precision) as s:
        s.set_mixed_load(dt=dt)
        s.step(n_inc)
        return np.array([h["S"][2] for h in s.history()])


def test_history_gradient_zero_misfit_and_fp32(lib, cuda):
    """A target equal to the model's own curve gives J = 0 and an exactly zero gradient (every
    increment's adjoint source vanishes, so no adjoint iteration runs).  A target that differs
    only in the last two increments leaves the first increments without a direct source; the
    FP32 adjoint then agrees with the FP64 one to the FP32 solve's accuracy."""
    from oracle.voronoi import label_rve

    from paper_2402_09996_gb300 import inputs, rve

    inp = inputs.make_inputs((12, 10, 16), 6, 0.5, seed=33)
    gid = label_rve(inp)
    n_inc, dt = 5, 0.5
    S32 = _history_S33(gid, inp.euler, n_inc, dt, rve.FP32)
    J, gp, ge, info = rve.history_gradient(gid, inp.euler, n_inc, dt, S32, precision=rve.FP32, checkpoint_every=2)
    assert J == 0.0
    assert np.all(gp == 0.0) and np.all(ge == 0.0)
    assert info["adjoint_iterations"] == 0
    S64 = _history_S33(gid, inp.euler, n_inc, dt, rve.FP64)
    target = S64.copy()
    target[-2:] *= 0.98
    J64, gp64, ge64, _ = rve.history_gradient(gid, inp.euler, n_inc, dt, target, precision=rve.FP64,
                                              checkpoint_every=2)
    J32, gp32, ge32, info32 = rve.history_gradient(gid, inp.euler, n_inc, dt, target, precision=rve.FP32,
                                                   checkpoint_every=2)
    assert info32["adjoint_iterations"] > 0
    assert abs(J32 - J64) < 1e-3 * J64
    assert np.max(np.abs(gp32 - gp64)) < 2e-3 * np.max(np.abs(gp64)), (gp32, gp64)
    assert np.max(np.abs(ge32 - ge64)) < 2e-3 * np.max(np.abs(ge64)), (ge32, ge64)


def test_history_gradient_storage_modes_agree(lib, cuda):
    """Keeping every increment's fields on the device (no replay) and checkpointing with
    replayed segments give the same misfit and gradient: the replays reproduce the forward
    increments exactly (deterministic kernels)."""
    from oracle.voronoi import label_rve

    from paper_2402_09996_gb300 import inputs, rve

    inp = inputs.make_inputs((8, 10, 12), 4, 0.5, seed=5)
    gid = label_rve(inp)
    n_inc, dt = 4, 0.5
    target = np.array([90.0, 180.0, 240.0, 270.0])
    ref = rve.history_gradient(gid, inp.euler, n_inc, dt, target, checkpoint_every=2)
    stored = rve.history_gradient(gid, inp.euler, n_inc, dt, target, checkpoint_every=None)
    auto_ck = rve.history_gradient(gid, inp.euler, n_inc, dt, target, checkpoint_every=None, memory_budget=0)
    assert stored[3]["stored_fields"] and not auto_ck[3]["stored_fields"]
    assert auto_ck[3]["checkpoints"] == [0, 2]
    for other in (stored, auto_ck):
        assert other[0] == ref[0]
        assert np.array_equal(other[1], ref[1]) and np.array_equal(other[2], ref[2])


def test_history_misfit_autograd_function(lib, cuda):
    """rve.HistoryMisfit as a torch.autograd.Function: the forward value is the history's
    misfit and backward hands back exactly the adjoint gradient, scaled by the incoming
    gradient."""
    import torch

    from oracle.voronoi import label_rve

    from paper_2402_09996_gb300 import inputs, rve

    inp = inputs.make_inputs((8, 10, 12), 4, 0.5, seed=8)
    gid = label_rve(inp)
    n_inc, dt = 3, 0.5
    target = np.array([95.0, 185.0, 245.0])
    base = rve.default_material().as_dict()
    p0 = np.array([base[k] for k in rve.PARAM_NAMES], dtype=np.float64)
    J, gp, ge, _ = rve.history_gradient(gid, inp.euler, n_inc, dt, target)
    params = torch.tensor(p0, requires_grad=True)
    euler = torch.tensor(inp.euler, dtype=torch.float64, requires_grad=True)
    config = {"grain_id": gid, "n_increments": n_inc, "dt": dt, "target": target}
    out = rve.HistoryMisfit.apply(params, euler, config)
    assert float(out.detach()) == J
    (3.0 * out).backward()
    assert np.array_equal(params.grad.numpy(), 3.0 * gp)
    assert np.array_equal(euler.grad.numpy(), 3.0 * ge)


def test_history_gradient_register_transform_grid(lib, cuda):
    """The adjoint on a grid whose x and y lines take the two-step register transforms
    (8 x 64 x 64, FP64): the gradient in r0_ord and Q_s against central differences of the
    forward solve."""
    from oracle.voronoi import label_rve

    from paper_2402_09996_gb300 import inputs, rve

    inp = inputs.make_inputs((8, 64, 64), 6, 0.5, seed=64)
    gid = label_rve(inp)
    n_inc, dt = 3, 0.5
    opts = dict(tol=1e-12, max_iter=3000)
    _, S0 = _history_J(gid, inp.euler, {}, np.zeros(n_inc), n_inc, dt, **opts)
    target = 0.97 * S0
    J, gp, _, _ = rve.history_gradient(gid, inp.euler, n_inc, dt, target, **opts)
    base = orc.Material()
    for name in ("r0_ord", "Q_s"):
        k = rve.PARAM_NAMES.index(name)
        p0 = getattr(base, name)
        h = 1e-5 * abs(p0)
        jp, _ = _history_J(gid, inp.euler, {name: p0 + h}, target, n_inc, dt, **opts)
        jm, _ = _history_J(gid, inp.euler, {name: p0 - h}, target, n_inc, dt, **opts)
        num = (jp - jm) / (2 * h)
        assert abs(num - gp[k]) <= 1e-4 * max(abs(num), abs(gp[k])) + 1e-9 * J / abs(p0), (name, num, gp[k])


def _oracle_fd_case():
    """6 x 8 x 10 grid, 3 parent grains all twinned (6 orientations), 3 increments of 1 s
    (0.3 % strain, slip and twinning active in increments 2 and 3), tolerance 1e-12: the
    oracle's <sigma_zz> curve, a target 3 % below it, and central differences (relative
    step 1e-4; 1e-4 rad for angles) of the oracle's misfit for the 9 parameters and two
    Bunge angles."""
    import oracle_jobs
    from oracle.voronoi import label_rve

    from paper_2402_09996_gb300 import inputs, rve

    inp = inputs.make_inputs((6, 8, 10), 3, 1.0, seed=12)
    gid = label_rve(inp)
    euler = inp.euler.copy()
    n_inc, dt, tol = 3, 1.0, 1e-12
    base = orc.Material()
    jobs = [(gid, euler, {}, n_inc, dt, tol)]
    steps = []
    for name in rve.PARAM_NAMES:
        p0 = getattr(base, name)
        h = 1e-4 * abs(p0)
        steps.append(("param", name, h))
        jobs += [(gid, euler, {name: p0 + h}, n_inc, dt, tol), (gid, euler, {name: p0 - h}, n_inc, dt, tol)]
    for g, a in ((0, 1), (3, 0)):  # a parent's Phi and a twin's phi1
        ep, em = euler.copy(), euler.copy()
        ep[g, a] += 1e-4
        em[g, a] -= 1e-4
        steps.append(("euler", (g, a), 1e-4))
        jobs += [(gid, ep, {}, n_inc, dt, tol), (gid, em, {}, n_inc, dt, tol)]
    res = oracle_jobs.run_parallel(jobs)
    target = 0.97 * res[0]
    J = lambda S: float(np.sum((S - target) ** 2))  # noqa: E731
    fd = {key: (J(res[1 + 2 * k]) - J(res[2 + 2 * k])) / (2 * h) for k, (_, key, h) in enumerate(steps)}
    return gid, euler, n_inc, dt, target, J(res[0]), fd


def test_history_gradient_matches_oracle_finite_differences(lib, cuda):
    """The adjoint gradient of a load history against the FP64 oracle: the FP64 GPU
    gradient (tolerance 1e-12) within 1e-4 of central differences of the oracle's own
    misfit for all 9 parameters and two Bunge angles, and the misfit itself equal to the
    oracle's; the FP32 gradient (FP32 forward and adjoint, tolerance 1e-6) against the same
    differences within 1e-4 relative (measured: at most 3.1e-5)."""
    from paper_2402_09996_gb300 import rve

    gid, euler, n_inc, dt, target, J_ref, fd = _oracle_fd_case()
    J, gp, ge, _ = rve.history_gradient(gid, euler, n_inc, dt, target, precision=rve.FP64, tol=1e-12,
                                        max_iter=3000)
    assert abs(J - J_ref) <= 1e-8 * J_ref, (J, J_ref)
    got = {name: gp[k] for k, name in enumerate(rve.PARAM_NAMES)}
    got.update({(0, 1): ge[0, 1], (3, 0): ge[3, 0]})
    for key, num in fd.items():
        assert abs(got[key] - num) <= 1e-4 * abs(num), (key, got[key], num)
    J32, gp32, ge32, _ = rve.history_gradient(gid, euler, n_inc, dt, target, precision=rve.FP32)
    got32 = {name: gp32[k] for k, name in enumerate(rve.PARAM_NAMES)}
    got32.update({(0, 1): ge32[0, 1], (3, 0): ge32[3, 0]})
    errs = {str(key): abs(got32[key] - num) / abs(num) for key, num in fd.items()}
    print("FP32 adjoint vs oracle central differences, relative error:", errs)
    assert abs(J32 - J_ref) <= 1e-3 * J_ref
    assert max(errs.values()) <= 1e-4, errs
