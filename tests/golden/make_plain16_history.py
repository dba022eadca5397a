"""Writes plain16_fp64_history.json: the FP64 oracle's full load history on the 16^3
workload (8 untwinned Voronoi grains, seed 0), 10 increments of 1 s at 1e-3/s uniaxial
strain rate with the other stresses held at zero, tolerance 1e-6 (Sec. 4 criterion).

Calls only the oracle and the seeded input generator; about three minutes on one core.
Run from the repository root:  python tests/golden/make_plain16_history.py
"""
import json
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import rve_oracle as orc  # noqa: E402
from oracle.voronoi import label_rve  # noqa: E402
from paper_2402_09996_gb300.inputs import workload_plain_16  # noqa: E402

N_INCREMENTS = 10
DT = 1.0


def main():
    inp = workload_plain_16()
    gid = label_rve(inp)
    rve = orc.OracleRVE(gid, inp.euler, orc.Material(), orc.Options())
    rve.set_load(orc.Load(dt=DT))
    out = []
    for _ in range(N_INCREMENTS):
        r = rve.step()
        out.append({
            "increment": r["increment"],
            "iterations": r["iterations"],
            "E": [float(x) for x in r["E"]],
            "S": [float(x) for x in r["S"]],
            "S_eq_of_mean": r["S_eq_of_mean"],
            "mean_S_eq": r["mean_S_eq"],
            "mean_f": r["mean_f"],
            "mean_v": r["mean_v"],
            "residuals": [[float(e), float(c)] for e, c in r["residuals"]],
        })
        print(r["increment"], r["iterations"], r["S"][2], flush=True)
    doc = {
        "what": "FP64 oracle load history, 16^3 plain workload (8 grains, seed 0, no twins)",
        "load": {"Edot_33": 1e-3, "dt": DT, "increments": N_INCREMENTS, "stress_free": [0, 1, 3, 4, 5]},
        "n_sub": orc.default_n_sub(DT),
        "tol": 1e-6,
        "history": out,
    }
    path = Path(__file__).with_name("plain16_fp64_history.json")
    path.write_text(json.dumps(doc, indent=1) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
