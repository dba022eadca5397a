"""Host-side checks of the C ABI library (no GPU needed): it builds for sm_103a, loads,
exports every entry point declared in include/rve.h, and refuses to run without a
device instead of falling back to the CPU."""
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent


def _declared():
    text = (ROOT / "include" / "rve.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rve_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("rve_create", "rve_set_material", "rve_set_mixed_load", "rve_step", "rve_get_effective",
              "rve_get_fields", "rve_save_state", "rve_load_state", "rve_last_error", "rve_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    import subprocess

    from paper_2402_09996_gb300 import rve

    out = subprocess.run(["nm", "-D", "--defined-only", str(rve.LIB_PATH)], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rve_[a-z0-9_]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    assert sorted(_declared()) == sorted(rve.EXPORTED)


def test_defaults_roundtrip(lib):
    from paper_2402_09996_gb300 import rve

    o = rve.default_options()
    assert (o.precision, o.green, o.n_sub, o.max_iter, o.fixed_iters, o.tol) == (0, 0, 0, 1000, 0, 1e-6)
    assert (o.graphs, o.autotune, o.y_tile, o.z_tile, o.batch_group) == (1, 1, 0, 0, 0)
    m = rve.default_material().as_dict()
    assert m["C33"] == 178000.0 and m["eta"] == 1e4 and m["h_off"] == 1.2 and m["Kc"] == 1.45


def test_no_cpu_fallback_without_device(lib):
    import torch

    from paper_2402_09996_gb300 import rve

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(rve.RVEError) as ei:
        rve.RVE(np.zeros((4, 4, 4), np.uint32), np.zeros((1, 3)), use_torch=False)
    assert ei.value.status == 2
