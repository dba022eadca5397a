"""Oracle runs that the parity tests fan out over spawned processes (test infrastructure:
each job calls only the FP64 oracle)."""
import numpy as np


def history_s33(job):
    """<sigma_zz> of every increment of an oracle load history.

    job = (grain_id (nz, ny, nx), euler (n_grains, 3), material overrides (dict),
    n_increments, dt, tol)."""
    from oracle import rve_oracle as orc

    gid, euler, mat_kw, n_inc, dt, tol = job
    r = orc.OracleRVE(np.asarray(gid, dtype=np.int64), euler, orc.Material(**mat_kw),
                      orc.Options(tol=tol, max_iter=3000))
    r.set_load(orc.Load(dt=dt))
    return np.array([rec["S"][2] for rec in r.run(n_inc)])


def run_parallel(jobs):
    """history_s33 of every job, one spawned process per job (up to the core count)."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor

    saved = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"
    try:
        with ProcessPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1)),
                                 mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(history_s33, jobs))
    finally:
        if saved is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = saved
