"""dp_neighbor_pairs_static: the pair build for callers that cannot allocate
device memory (an engine that owns all device memory through its own pool,
or a time-critical loop where cudaMalloc/cudaFree must not run).  Its
output must equal the allocating entry point's, row set for row set, on
consecutive calls that reuse the library's fixed scratch array.  This file
is collected last so that a stop at the first failure has run every other
test first."""
import numpy as np
import pytest

from paper_2201_01446_gb300 import inputs

pytestmark = pytest.mark.gpu


def _sorted(a):
    return a[np.lexsort(a.T[::-1])]


def test_static_pairs_equal_allocating_entry_point(cu_model_path):
    torch = pytest.importorskip("torch")
    from paper_2201_01446_gb300 import dp
    h = dp.dp_create(cu_model_path, 1, 8.0, 0.5, [256], stream=None)
    try:
        cases = [(5, 0.05, 10.0, 1), ((4, 6, 5), 0.2, 8.0, 2), (3, 0.3, 8.0, 3)]
        for ncell, sigma, rlist, seed in cases:  # consecutive calls share the scratch
            x, _, box = inputs.fcc_copper(ncell, sigma=sigma, seed=seed)
            x = x + np.array([-2.5, 11.0, 0.75])
            ref = _sorted(dp.dp_neighbor_pairs(h, x, box, rlist))
            got = dp.dp_neighbor_pairs_static(torch.tensor(x, device="cuda"), box, rlist)
            torch.cuda.synchronize()
            got = _sorted(got.cpu().numpy())
            assert got.shape == ref.shape and len(ref) > 0
            assert np.array_equal(got, ref)
    finally:
        dp.dp_destroy(h)


def test_static_pairs_reject_beyond_capacity():
    torch = pytest.importorskip("torch")
    from paper_2201_01446_gb300 import dp
    x = torch.zeros((65537, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(dp.DPError) as e:
        dp.dp_neighbor_pairs_static(x, np.diag([100.0, 100.0, 100.0]), 8.0)
    assert e.value.code == 12
    # too many cells for the fixed array: a huge box at a small cutoff
    y = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(dp.DPError) as e:
        dp.dp_neighbor_pairs_static(y, np.diag([1000.0, 1000.0, 1000.0]), 2.0)
    assert e.value.code == 12
