"""rve_step_batch: several RVEs of different sizes and precisions stepped concurrently
give exactly the results of stepping each alone; a failing member is isolated."""
import numpy as np
import pytest

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
