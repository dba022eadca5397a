"""Checks the sampled voxels that `bench.py --workload precision256 --dump-sample PATH`
writes against the oracle's material-point update (Sec. 3 law with the Sec. 4 regularised
rates, RK4 along the linear strain path of the increment).

For each precision, from the committed state of the sampled voxels before its last
increment to the converged strain after it, the oracle recomputes the stress, plastic
strain, accumulated slip and kinematic variables; the largest relative errors against
the GPU's committed values are printed as one JSON line.  The grid is too large for the
oracle's full solve; this per-voxel check holds at any size.

Run from the repository root:  python tests/check_material_point_sample.py PATH
"""
import json
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))
sys.path.insert(0, str(ROOT / "tests"))

from helpers import six_to_tensor  # noqa: E402
from oracle import rve_oracle as orc  # noqa: E402


def check(path):
    d = np.load(path)
    euler, grain, dt = d["euler"], d["grain"], float(d["dt"])
    out = {}
    for name in ("fp64", "fp32"):
        R = np.stack([orc.bunge_rotation(euler[g]) for g in grain])
        if name == "fp32":
            R = R.astype(np.float32).astype(np.float64)  # the rotation as the float kernel sees it
        b = lambda key: d[f"{name}_before_{key}"]  # noqa: E731
        a = lambda key: d[f"{name}_after_{key}"]  # noqa: E731
        sig_ref, ep_ref, v_ref, al_ref = orc.material_point_increment(
            orc.Material(), R, six_to_tensor(b("eps")), six_to_tensor(a("eps")), six_to_tensor(b("eps_p")),
            b("v").T, b("alpha").T, dt, int(d[f"{name}_n_sub"]))
        sig = six_to_tensor(a("sigma"))
        err_sig = np.linalg.norm(sig - sig_ref, axis=(1, 2)) / np.linalg.norm(sig_ref, axis=(1, 2))
        scale = lambda r: max(float(np.max(np.abs(r))), 1e-300)  # noqa: E731
        out[name] = {
            "sigma_max_rel_per_voxel": float(np.max(err_sig)),
            "eps_p_max_rel": float(np.max(np.abs(six_to_tensor(a("eps_p")) - ep_ref)) / scale(ep_ref)),
            "v_max_rel": float(np.max(np.abs(a("v").T - v_ref)) / scale(v_ref)),
            "alpha_max_rel": float(np.max(np.abs(a("alpha").T - al_ref)) / scale(al_ref)),
            "flowing_fraction": float(np.mean(np.any(v_ref > b("v").T, axis=1))),
            "samples": int(len(grain)),
        }
    return out


if __name__ == "__main__":
    print(json.dumps(check(sys.argv[1])))
