"""Shared test helpers: tensor layout conversions (no method arithmetic)."""
import numpy as np

IDX6 = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def six_to_tensor(a6):
    """(6, ...) tensor components (11,22,33,23,13,12) -> (..., 3, 3)."""
    a6 = np.asarray(a6)
    out = np.zeros(a6.shape[1:] + (3, 3))
    for c, (i, j) in enumerate(IDX6):
        out[..., i, j] = a6[c]
        out[..., j, i] = a6[c]
    return out


def tensor_to_six(t):
    """(..., 3, 3) -> (6, ...)."""
    return np.stack([t[..., i, j] for i, j in IDX6], axis=0)


def rel_err(a, b):
    """max |a - b| / max |b| (real or complex)."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))
