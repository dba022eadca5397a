"""The seeded input generator: published SplitMix64 vectors, Haar sampling, twin draws."""
import math

import numpy as np

from oracle import rve_oracle as orc
from paper_2402_09996_gb300 import inputs


def test_splitmix64_reference_vectors():
    # first outputs of SplitMix64 seeded with 1234567 (reference C implementation)
    r = inputs.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(3)] == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_uniforms_in_unit_interval_and_deterministic():
    a = inputs.SplitMix64(7).uniforms(1000)
    b = inputs.SplitMix64(7).uniforms(1000)
    assert np.array_equal(a, b) and a.min() >= 0.0 and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.03


def test_haar_orientations():
    inp = inputs.make_inputs((8, 8, 8), 4000, 0.0, seed=1)
    e = inp.euler[:4000]
    assert np.all((e[:, 0] >= 0) & (e[:, 0] < 2 * np.pi) & (e[:, 1] >= 0) & (e[:, 1] <= np.pi))
    # Haar measure: cos(Phi) uniform on [-1, 1] -> mean 0, variance 1/3
    c = np.cos(e[:, 1])
    assert abs(c.mean()) < 0.03 and abs(c.var() - 1 / 3) < 0.02
    # the crystal c axis is uniform on the sphere
    R = orc.bunge_rotation(e)
    assert np.abs(R[:, :, 2].mean(axis=0)).max() < 0.03


def test_twin_is_half_turn_about_the_plane_normal():
    inp = inputs.make_inputs((8, 8, 8), 50, 0.5, seed=5)
    n = inp.n_parent
    assert 10 < inp.twinned.sum() < 40
    Rp = orc.bunge_rotation(inp.euler[:n])
    Rt = orc.bunge_rotation(inp.euler[n:])
    for p in range(n):
        if not inp.twinned[p]:
            assert np.array_equal(inp.euler[n + p], inp.euler[p])
            continue
        ns = inp.twin_normal[p]
        # the normal is a {111} plane normal of the parent, expressed in the sample frame
        nc = Rp[p].T @ ns
        assert np.allclose(np.abs(nc), 1 / math.sqrt(3))
        # misorientation R_t R_p^T is a 180 degree rotation about ns
        M = Rt[p] @ Rp[p].T
        assert np.allclose(M, 2 * np.outer(ns, ns) - np.eye(3), atol=1e-12)
