"""Element-wise parity of the CUDA steps with the FP64 oracle: the 3-D FFT used by the
Green-operator step and the per-voxel constitutive update (Sec. 3 / Sec. 4)."""
import numpy as np
import pytest

from helpers import rel_err, six_to_tensor, tensor_to_six
from oracle import rve_oracle as orc

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4), (16, 16, 16), (6, 10, 12), (12, 20, 30), (5, 9, 16), (8, 6, 96), (4, 4, 160), (3, 128, 4),
          (1, 4, 6), (1, 1, 8), (2, 1, 2)]


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
