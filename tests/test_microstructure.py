"""The paper's microstructure model (Sec. 2.1-2.3) as drawn by inputs.paper_microstructure:
each rule of the model checked on its output (CPU, oracle labeller)."""
import math

import numpy as np
import pytest

from oracle import rve_oracle as orc
from oracle.voronoi import label_rve
from paper_2402_09996_gb300 import inputs

SHAPE = (40, 36, 48)


@pytest.fixture(scope="module")
def neigh():
    return inputs.paper_microstructure(SHAPE, label_rve, n_expected=70, r_hard_vox=4.0, p_neigh=1.0, p_incl=0.0,
                                       seed=11)


@pytest.fixture(scope="module")
def incl():
    return inputs.paper_microstructure(SHAPE, label_rve, n_expected=70, r_hard_vox=4.0, p_neigh=0.0, p_incl=1.0,
                                       seed=12)


def _rot(e):
    return orc.bunge_rotation(np.asarray(e))


def test_poisson_draw_has_poisson_moments():
    rng = inputs.SplitMix64(5)
    x = np.array([inputs.poisson(rng, 30.0) for _ in range(4000)])
    assert abs(x.mean() - 30.0) < 0.35  # 4 standard errors
    assert abs(x.var() / 30.0 - 1.0) < 0.1


def test_matern_hardcore_distance_and_intensity():
    r = 0.06
    counts = []
    for s in range(12):
        pts = inputs.matern_hardcore_seeds(inputs.SplitMix64(100 + s), 150.0, r)
        d = pts[:, None, :] - pts[None, :, :]
        d -= np.round(d)
        dist = np.sqrt(np.sum(d * d, axis=-1)) + np.eye(len(pts))
        assert dist.min() >= r
        counts.append(len(pts))
    # type II thinning with the solved parent intensity keeps 150 points on average
    assert abs(np.mean(counts) - 150.0) < 4.0 * math.sqrt(150.0 / 12) + 3.0


def test_neighbouring_twins_follow_the_model(neigh):
    m = neigh
    n_vor = m.seeds.shape[0]
    assert m.n_grains == n_vor and not m.inclusions
    assert 0 < len(m.pairs) <= n_vor // 2
    adj = {tuple(p) for p in inputs.grain_adjacency(m.gid).tolist()}
    used = set()
    theta = math.radians(inputs.TWIN_MISORIENTATION_DEG)
    for k, l_, hi, sign in m.pairs:
        assert (min(k, l_), max(k, l_)) in adj  # a contiguous pair
        assert k not in used and l_ not in used  # no grain twice: no twin chains
        used |= {k, l_}
        Rk, Rl = _rot(m.euler[k]), _rot(m.euler[l_])
        d = m.seeds[l_] - m.seeds[k]
        d -= np.round(d)
        nrm = sign * d / np.linalg.norm(d)  # normal of the joint Voronoi facet
        assert np.allclose(Rk @ inputs.HABIT_NORMALS[hi], nrm, atol=1e-9)  # habit plane in the facet
        M = Rk.T @ Rl  # misorientation in the crystal frame of k
        assert abs((np.trace(M) - 1.0) / 2.0 - math.cos(theta)) < 1e-9
        assert np.allclose(M @ inputs.HABIT_AXES[hi], inputs.HABIT_AXES[hi], atol=1e-9)  # about [100] / [010]


def test_inclusion_twins_follow_the_model(incl):
    m = incl
    n_vor = m.seeds.shape[0]
    base = label_rve(inputs.RVEInputs(SHAPE, m.seeds, np.zeros((2 * n_vor, 3)), np.zeros(n_vor, np.uint8),
                                      np.zeros((n_vor, 3))))
    assert len(m.inclusions) == n_vor  # p_incl = 1
    assert m.n_grains == n_vor + len(m.inclusions)
    nz, ny, nx = SHAPE
    dims = np.array([nx, ny, nz], dtype=float)
    theta = math.radians(inputs.TWIN_MISORIENTATION_DEG)
    boundary = np.zeros(SHAPE, dtype=bool)
    for ax in range(3):
        boundary |= base != np.roll(base, 1, axis=ax)
        boundary |= base != np.roll(base, -1, axis=ax)
    for g, child, ai, x, thick in m.inclusions:
        parent_vox = base == g
        child_vox = m.gid == child
        assert np.all(parent_vox[child_vox])  # I is a subset of G
        xi = x.astype(int)
        assert parent_vox[xi[2], xi[1], xi[0]] and boundary[xi[2], xi[1], xi[0]]  # x on the boundary of G
        ved = (6.0 * parent_vox.sum() / math.pi) ** (1.0 / 3.0)
        assert 0.1 * ved - 1e-9 <= thick <= 0.3 * ved + 1e-9
        Rg, Rc = _rot(m.euler[g]), _rot(m.euler[child])
        nrm = Rg @ inputs.HABIT_NORMALS[ai]
        zz, yy, xx = np.nonzero(parent_vox)
        d = np.stack([xx, yy, zz], axis=1) - x
        d -= dims * np.round(d / dims)
        slab = np.abs(d @ nrm) <= 0.5 * thick
        # exactly the parent's voxels inside the slab belong to the inclusion
        assert np.array_equal(child_vox[zz, yy, xx], slab)
        M = Rg.T @ Rc
        assert abs((np.trace(M) - 1.0) / 2.0 - math.cos(theta)) < 1e-9
        assert np.allclose(M @ inputs.HABIT_AXES[ai], inputs.HABIT_AXES[ai], atol=1e-9)


def test_paper_microstructure_is_reproducible():
    a = inputs.paper_microstructure((16, 16, 16), label_rve, n_expected=12, r_hard_vox=2.0, p_neigh=1.0, p_incl=0.5,
                                    seed=4)
    b = inputs.paper_microstructure((16, 16, 16), label_rve, n_expected=12, r_hard_vox=2.0, p_neigh=1.0, p_incl=0.5,
                                    seed=4)
    assert np.array_equal(a.gid, b.gid) and np.array_equal(a.euler, b.euler)
