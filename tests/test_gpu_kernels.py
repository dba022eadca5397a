"""Element-wise parity of the CUDA steps with the FP64 oracle: the 3-D FFT used by the
Green-operator step and the per-voxel constitutive update (Sec. 3 / Sec. 4)."""
import numpy as np
import pytest

from helpers import rel_err, six_to_tensor, tensor_to_six
from oracle import rve_oracle as orc

pytestmark = pytest.mark.gpu

# (nz, ny, nx): Stockham lengths, and lines of 64, 96, 128, 160 and 256 points (register
# two-step transforms) in each direction, with kx ranges split into several uneven chunks
SHAPES = [(4, 4, 4), (16, 16, 16), (6, 10, 12), (12, 20, 30), (5, 9, 16), (8, 6, 96), (4, 4, 160), (3, 128, 4),
          (1, 4, 6), (1, 1, 8), (2, 1, 2), (64, 5, 6), (4, 96, 8), (256, 2, 4), (2, 4, 256), (160, 2, 2),
          (3, 64, 64), (8, 128, 96), (64, 3, 256), (3, 5, 128)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fft_r2c_matches_oracle(lib, cuda, shape, prec):
    import torch

    from paper_2402_09996_gb300 import rve

    p = rve.FP64 if prec == "fp64" else rve.FP32
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal((3,) + shape)
    xt = torch.tensor(x, device=cuda, dtype=torch.float64 if p == rve.FP64 else torch.float32)
    got = rve.fft_r2c(xt, p).cpu().numpy()
    ref = orc.rfft3(x.astype(np.float32) if p == rve.FP32 else x)
    tol = 1e-13 if p == rve.FP64 else 2e-6
    assert got.shape == ref.shape
    assert rel_err(got, ref) < tol
    # unnormalised inverse brings back N x
    cdt = torch.complex128 if p == rve.FP64 else torch.complex64
    back = rve.fft_c2r(torch.tensor(ref, device=cuda, dtype=cdt), shape[2], p).cpu().numpy()
    assert rel_err(back / np.prod(shape), x) < (1e-13 if p == rve.FP64 else 2e-6)


def _random_material_points(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    e = rng.uniform(0, 2 * np.pi, size=(n, 3))
    e[:, 1] = np.arccos(rng.uniform(-1, 1, size=n))
    R = orc.bunge_rotation(e)
    eps_n = rng.normal(scale=1.5e-3, size=(n, 3, 3)) * scale
    eps_n = 0.5 * (eps_n + eps_n.transpose(0, 2, 1))
    d = rng.normal(scale=1.0e-3, size=(n, 3, 3)) * scale
    eps = eps_n + 0.5 * (d + d.transpose(0, 2, 1))
    quiet = rng.uniform(size=n) < 0.3  # small strains: a share of elastic voxels
    eps_n[quiet] *= 0.1
    eps[quiet] *= 0.1
    ep = rng.normal(scale=3e-4, size=(n, 3, 3))
    ep = 0.5 * (ep + ep.transpose(0, 2, 1))
    ep -= np.trace(ep, axis1=1, axis2=2)[:, None, None] * np.eye(3) / 3
    v = rng.uniform(0, 2e-3, size=(n, 16))
    v[:, 12:] *= 0.1
    al = rng.uniform(-1e-3, 1e-3, size=(n, 12))
    return R, eps_n, eps, ep, v, al


@pytest.mark.parametrize("prec,n,dt", [("fp64", 777, 1.0), ("fp32", 1000, 0.5), ("fp64", 1, 0.5)])
def test_material_point_matches_oracle(lib, cuda, prec, n, dt):
    import torch

    from paper_2402_09996_gb300 import rve

    p = rve.FP64 if prec == "fp64" else rve.FP32
    tdt = torch.float64 if p == rve.FP64 else torch.float32
    R, eps_n, eps, ep, v, al = _random_material_points(n, 7 + n)
    if p == rve.FP32:  # the oracle sees exactly the inputs the float kernel sees
        R, eps_n, eps, ep, v, al = (a.astype(np.float32).astype(np.float64) for a in (R, eps_n, eps, ep, v, al))
    nsub = orc.default_n_sub(dt)
    mat = orc.Material()
    sig_ref, ep_ref, v_ref, al_ref = orc.material_point_increment(mat, R, eps_n, eps, ep, v, al, dt, nsub)
    state = np.concatenate([tensor_to_six(ep), v.T, al.T], axis=0)
    to_dev = lambda a: torch.tensor(np.ascontiguousarray(a), device=cuda, dtype=tdt)  # noqa: E731
    st = to_dev(state)
    sig = rve.material_point(to_dev(R.reshape(n, 9)), to_dev(tensor_to_six(eps_n)), to_dev(tensor_to_six(eps)), st,
                             dt, nsub, p).cpu().numpy()
    st = st.cpu().numpy()
    tol = 1e-10 if p == rve.FP64 else 2e-4
    assert rel_err(six_to_tensor(sig), sig_ref) < tol
    assert rel_err(six_to_tensor(st[:6]), ep_ref) < tol
    assert rel_err(st[6:22].T, v_ref) < tol
    assert rel_err(st[22:].T, al_ref) < tol
    # the mix must contain both elastic and plastic voxels
    if n > 100:
        active = np.any(np.abs(v_ref - v) > 0, axis=1)
        assert 0.05 < active.mean() < 0.999


PAPER_SET = dict(C33=183000.0, r0_ord=130.0, r0_sup=200.0, r0_twin=130.0, K=104.0, Kt=104.0, n=6.42, nt=6.42,
                 Q_s=9.57, Q_b=10.5, Kc=1.45, fm=0.8, eta=1.0e4, c=0.0, d=0.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("which", ["paper", "int5_7", "eta0"])
def test_material_point_other_rate_laws_match_oracle(lib, cuda, prec, which):
    """The branch-free solve with real exponents (the paper's n = nt = 6.42; integer n = 5,
    nt = 7) and the generic solve without regularisation (eta = 0; a slow Norton law, K =
    3000 MPa s^(1/n), keeps the explicit RK4 stable at these increments) against the oracle."""
    import dataclasses

    import torch

    from paper_2402_09996_gb300 import rve

    mat_kw = {"paper": PAPER_SET, "int5_7": dict(n=5.0, nt=7.0),
              "eta0": dict(eta=0.0, n=2.5, nt=2.5, K=3000.0, Kt=3000.0)}[which]
    p = rve.FP64 if prec == "fp64" else rve.FP32
    tdt = torch.float64 if p == rve.FP64 else torch.float32
    n = 600
    R, eps_n, eps, ep, v, al = _random_material_points(n, 31, scale=3.0 if which == "paper" else 1.0)
    if p == rve.FP32:
        R, eps_n, eps, ep, v, al = (a.astype(np.float32).astype(np.float64) for a in (R, eps_n, eps, ep, v, al))
    dt = 0.5
    nsub = orc.default_n_sub(dt)
    mat = dataclasses.replace(orc.Material(), **mat_kw)
    sig_ref, ep_ref, v_ref, al_ref = orc.material_point_increment(mat, R, eps_n, eps, ep, v, al, dt, nsub)
    state = np.concatenate([tensor_to_six(ep), v.T, al.T], axis=0)
    to_dev = lambda a: torch.tensor(np.ascontiguousarray(a), device=cuda, dtype=tdt)  # noqa: E731
    st = to_dev(state)
    sig = rve.material_point(to_dev(R.reshape(n, 9)), to_dev(tensor_to_six(eps_n)), to_dev(tensor_to_six(eps)), st,
                             dt, nsub, p, **mat_kw).cpu().numpy()
    st = st.cpu().numpy()
    tol = 1e-10 if p == rve.FP64 else 2e-4
    assert rel_err(six_to_tensor(sig), sig_ref) < tol
    assert rel_err(six_to_tensor(st[:6]), ep_ref) < tol
    assert rel_err(st[6:22].T, v_ref) < tol
    assert rel_err(st[22:].T, al_ref) < tol
    active = np.any(np.abs(v_ref - v) > 0, axis=1)
    assert 0.05 < active.mean() < 0.999
