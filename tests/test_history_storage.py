"""Host logic of the load-history adjoint: how the history is kept (CPU)."""
import pytest

from paper_2402_09996_gb300 import rve


def test_explicit_checkpoint_interval_is_kept():
    assert rve.history_storage(30, 96 ** 3, 5, memory_budget=1 << 60) == (False, 5)
    assert rve.history_storage(30, 96 ** 3, 1, memory_budget=0) == (False, 1)
    with pytest.raises(ValueError):
        rve.history_storage(30, 96 ** 3, 0, memory_budget=0)


def test_fields_kept_when_they_fit():
    nvox, n = 96 ** 3, 30
    need = 8 * 40 * nvox * (n + 1)  # strain 6 + state 34 values, FP64, n + 1 time levels
    assert rve.history_storage(n, nvox, None, memory_budget=need) == (True, n)
    assert rve.history_storage(n, nvox, None, memory_budget=need - 1)[0] is False


def test_checkpoint_fallback_is_ceil_sqrt():
    for n, k in [(1, 1), (2, 2), (4, 2), (5, 3), (9, 3), (10, 4), (30, 6), (1000, 32)]:
        assert rve.history_storage(n, 16, None, memory_budget=0) == (False, k), n
