"""rve_step_batch: several RVEs of different sizes and precisions stepped concurrently
give exactly the results of stepping each alone; a failing member is isolated.  Handles
of one precision, material and load run as one group (one launch per pass over all
members): the same holds there, and a small member equals the oracle."""
import numpy as np
import pytest

from oracle import rve_oracle as orc
from oracle.voronoi import label_rve

pytestmark = pytest.mark.gpu


def _members():
    from paper_2402_09996_gb300 import inputs, rve

    out = []
    inp = inputs.make_inputs((12, 10, 6), 5, 0.5, seed=42)  # ragged, twinned
    out.append((label_rve(inp), inp.euler, rve.FP64, 0.5))
    inp = inputs.workload_plain_16()
    out.append((label_rve(inp), inp.euler, rve.FP64, 1.0))
    inp = inputs.make_inputs((24, 20, 32), 9, 0.5, seed=7)
    out.append((label_rve(inp), inp.euler, rve.FP32, 0.5))
    gid = np.zeros((8, 8, 8), dtype=np.uint32)
    gid[:, :, 4:] = 1
    out.append((gid, np.array([[0.3, 0.9, 1.7], [2.1, 1.2, 0.4]]), rve.FP32, 0.5))
    return out


def _make(member, **kw):
    from paper_2402_09996_gb300 import rve

    gid, euler, prec, dt = member
    s = rve.RVE(np.asarray(gid, dtype=np.uint32), euler, precision=prec, **kw)
    s.set_mixed_load(dt=dt)
    return s


def test_batch_equals_sequential(lib, cuda):
    from paper_2402_09996_gb300 import rve

    members = _members()
    alone = []
    for m in members:
        with _make(m) as s:
            s.step(3)
            alone.append((s.history(), s.field(rve.FIELD_STRESS), s.field(rve.FIELD_V)))
    solvers = [_make(m) for m in members]
    try:
        its = rve.step_batch(solvers, 2)
        its += rve.step_batch(solvers[::-1], 1)  # order of the handles does not matter
        assert its == sum(h["iterations"] for hist, _, _ in alone for h in hist)
        for s, (hist, sig, v) in zip(solvers, alone):
            got = s.history()
            assert len(got) == 3
            for g, r in zip(got, hist):
                assert g["iterations"] == r["iterations"]
                for key in ("E", "S"):
                    assert np.array_equal(g[key], r[key])  # deterministic kernels: bit-identical
                for key in ("residual", "stress_residual", "mean_S_eq", "mean_v", "mean_f"):
                    assert g[key] == r[key]
            assert np.array_equal(s.field(rve.FIELD_STRESS), sig)
            assert np.array_equal(s.field(rve.FIELD_V), v)
    finally:
        for s in solvers:
            s.close()


def test_batch_isolates_a_failing_member(lib, cuda):
    from paper_2402_09996_gb300 import rve

    members = _members()
    good = _make(members[1])
    bad = _make(members[0], max_iter=3)  # cannot reach 1e-6 in 3 iterations
    try:
        with pytest.raises(rve.RVEError) as ei:
            rve.step_batch([good, bad], 2)
        assert ei.value.status == rve.STATUS_CODES["RVE_ERR_NOT_CONVERGED"]
        assert ei.value.index == 1
        assert "handle 1" in str(ei.value)
        assert len(good.history()) == 2  # the others still run every increment
        assert len(bad.history()) == 0  # the failing one keeps its committed state
        # the good member's result equals a sequential run
        with _make(members[1]) as ref:
            ref.step(2)
            assert np.array_equal(ref.history()[-1]["S"], good.history()[-1]["S"])
        # duplicate handles are rejected before any work
        with pytest.raises(rve.RVEError) as ei:
            rve.step_batch([good, good], 1)
        assert ei.value.status == rve.STATUS_CODES["RVE_ERR_INVALID_ARG"]
        assert len(good.history()) == 2
    finally:
        good.close()
        bad.close()


def _group_members(prec):
    """RVEs of one precision and load whose x, y and z lines take every transform kind:
    Stockham (radix 2/3/5, ragged), and the register splits 64, 96, 128 and 160."""
    from paper_2402_09996_gb300 import inputs

    shapes = [(12, 10, 6), (24, 20, 32), (16, 12, 64), (8, 96, 10), (160, 6, 8), (6, 128, 12)]
    return [(label_rve(inp), inp.euler) for inp in
            (inputs.make_inputs(sh, 5, 0.5, seed=17 + k) for k, sh in enumerate(shapes))]


def _compare_exact(got, ref):
    assert len(got) == len(ref)
    for g, r in zip(got, ref):
        assert g["iterations"] == r["iterations"]
        for key in ("E", "S"):
            assert np.array_equal(g[key], r[key])
        for key in ("residual", "stress_residual", "mean_S_eq", "mean_v", "mean_f"):
            assert g[key] == r[key]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_grouped_batch_equals_sequential_and_oracle(lib, cuda, prec):
    """Six RVEs stepped as one group (one launch per pass over all of them, lockstep
    iterations) give bit for bit the results of stepping each alone; in FP64 the ragged
    6 x 10 x 12 member also matches the oracle's history directly (1e-8)."""
    from paper_2402_09996_gb300 import rve

    P = rve.FP32 if prec == "fp32" else rve.FP64
    members = _group_members(prec)
    alone = []
    for gid, euler in members:
        with rve.RVE(gid, euler, precision=P) as s:
            s.set_mixed_load(dt=0.5)
            s.step(3)
            alone.append((s.history(), s.field(rve.FIELD_STRESS), s.field(rve.FIELD_V)))
    solvers = []
    try:
        for gid, euler in members:
            s = rve.RVE(gid, euler, precision=P, batch_group=True)
            s.set_mixed_load(dt=0.5)
            solvers.append(s)
        assert rve.batch_grouped(solvers)
        its = rve.step_batch(solvers, 2)
        its += rve.step_batch(solvers[::-1], 1)
        assert its == sum(h["iterations"] for hist, _, _ in alone for h in hist)
        for s, (hist, sig, v) in zip(solvers, alone):
            _compare_exact(s.history(), hist)
            assert np.array_equal(s.field(rve.FIELD_STRESS), sig)
            assert np.array_equal(s.field(rve.FIELD_V), v)
        got_small = solvers[0].history()
    finally:
        for s in solvers:
            s.close()
    if P == rve.FP64:
        gid, euler = members[0]
        ref = orc.OracleRVE(np.asarray(gid, dtype=np.int64), euler, orc.Material(), orc.Options())
        ref.set_load(orc.Load(dt=0.5))
        ref.run(3)
        for g, r in zip(got_small, ref.history):
            assert g["iterations"] == r["iterations"]
            assert np.max(np.abs(g["S"] - r["S"])) < 1e-8 * np.max(np.abs(r["S"]))
            assert abs(g["mean_v"] - r["mean_v"]) <= 1e-8 * abs(r["mean_v"]) + 1e-15


def test_grouped_batch_isolates_a_failing_member_and_mixed_batches_use_streams(lib, cuda):
    """In a group, a member that hits its iteration cap keeps its committed state and
    leaves the group; the others run every increment, exactly as alone.  Handles of
    different precisions or loads, or with batch_group off (the default), are not grouped."""
    from paper_2402_09996_gb300 import rve

    (g0, e0), (g1, e1) = _group_members("fp64")[:2]
    good = rve.RVE(g1, e1, precision=rve.FP64, batch_group=True)
    bad = rve.RVE(g0, e0, precision=rve.FP64, max_iter=3, batch_group=True)
    other = rve.RVE(g0, e0, precision=rve.FP32, batch_group=True)
    loose = rve.RVE(g0, e0, precision=rve.FP64)  # batch_group off (the default)
    try:
        for s in (good, bad, other, loose):
            s.set_mixed_load(dt=0.5)
        assert rve.batch_grouped([good, bad])
        assert not rve.batch_grouped([good, other]) and not rve.batch_grouped([good, loose])
        assert not rve.batch_grouped([good])
        with pytest.raises(rve.RVEError) as ei:
            rve.step_batch([good, bad], 2)
        assert ei.value.status == rve.STATUS_CODES["RVE_ERR_NOT_CONVERGED"]
        assert ei.value.index == 1
        assert len(good.history()) == 2 and len(bad.history()) == 0
        with rve.RVE(g1, e1, precision=rve.FP64) as ref:
            ref.set_mixed_load(dt=0.5)
            ref.step(2)
            _compare_exact(good.history(), ref.history())
        other.set_mixed_load(dt=1.0)
        bad.set_mixed_load(dt=1.0)
        assert not rve.batch_grouped([good, bad])  # different loads
    finally:
        for s in (good, bad, other, loose):
            s.close()
