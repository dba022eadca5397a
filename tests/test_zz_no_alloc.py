"""The labelling entry point that allocates no device memory (for callers that own all
device memory or cannot afford the synchronisation of cudaMalloc/cudaFree) must give
exactly the labels of the allocating entry point, also on consecutive calls that share
its static scratch, and must refuse parent counts above its fixed maximum."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_labels_equal_allocating_entry_point_on_consecutive_calls(lib, cuda):
    import torch

    from paper_2402_09996_gb300 import inputs, rve

    cases = [((20, 24, 16), 40, 0.5, 3), ((20, 24, 16), 40, 0.5, 3), ((16, 18, 30), 12, 1.0, 8)]
    for shape, n, p, seed in cases:
        inp = inputs.make_inputs(shape, n, p, seed)
        ref = rve.label_voronoi(inp)
        out = torch.full(shape, -1, dtype=torch.int32, device=cuda)
        rve.label_voronoi_noalloc(inp, out)
        got = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, ref)  # labels are integers: bit-exact
        assert np.any(got >= n) == bool(np.any(inp.twinned))


def test_noalloc_rejects_more_parents_than_its_scratch_holds(lib, cuda):
    import torch

    from paper_2402_09996_gb300 import inputs, rve

    big = inputs.make_inputs((4, 4, 4), rve.NOALLOC_MAX_PARENTS + 1, 0.0, seed=1)
    out = torch.empty((4, 4, 4), dtype=torch.int32, device=cuda)
    with pytest.raises(rve.RVEError) as ei:
        rve.label_voronoi_noalloc(big, out)
    assert ei.value.status == 1
    assert "maximum" in str(ei.value)


def test_noalloc_wrapper_refuses_wrong_output_tensors(lib, cuda):
    import torch

    from paper_2402_09996_gb300 import inputs, rve

    inp = inputs.make_inputs((8, 8, 8), 5, 0.5, seed=2)
    for bad in (torch.empty((8, 8, 8), dtype=torch.int64, device=cuda),
                torch.empty((8, 8, 16), dtype=torch.int32, device=cuda)[:, :, ::2],
                torch.empty((8, 8, 8), dtype=torch.int32)):
        with pytest.raises(ValueError):
            rve.label_voronoi_noalloc(inp, bad)
