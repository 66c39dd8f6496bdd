"""dp_neighbor_pairs_static: the pair build for callers that cannot allocate
device memory (an engine that owns all device memory through its own pool,
or a time-critical loop where cudaMalloc/cudaFree must not run).  Its rows
must equal the oracle's brute-force / cell-list pair sets and the allocating
entry point's, on consecutive calls that reuse the library's fixed scratch
array (a many-cell grid before smaller ones, so stale cell data of a larger
call would show), including pairs within 1e-7 A of the cutoff, a call whose
capacity is smaller than the pair count, and a count past 2^31.  This file
is collected last so that a stop at the first failure has run every other
test first."""
import numpy as np
import pytest

import oracle
from paper_2201_01446_gb300 import inputs

pytestmark = pytest.mark.gpu


def _sorted(a):
    return a[np.lexsort(a.T[::-1])]


def _band_case():
    # 40 atoms within 1e-7 A of the cutoff around one centre: the FP64
    # recheck of the FP32 band decides every one of them
    box = np.diag([30.0, 30.0, 30.0])
    rng = np.random.default_rng(5)
    xs = [np.array([15.0, 15.0, 15.0])]
    for _ in range(40):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        xs.append(xs[0] + d * (8.0 + rng.choice([-1, 1]) * rng.uniform(0, 1e-7)))
    return np.array(xs), box, 8.0


def _cases():
    out = []
    # 8^3 FCC cells (29.07 A) at rlist 4: 7 cells per axis, interior stencil
    x, _, box = inputs.fcc_copper(8, sigma=0.1, seed=4)
    out.append((x + np.array([3.3, -40.0, 0.5]), box, 4.0, "Cu 2048, 7^3 cells"))
    x, _, box = inputs.fcc_copper((4, 6, 5), sigma=0.2, seed=2)
    out.append((x + np.array([-2.5, 11.0, 0.75]), box, 8.0, "Cu 480, 1x2x2 cells"))
    x, _, box = inputs.fcc_copper(3, sigma=0.3, seed=3)
    out.append((x, box, 8.0, "Cu 108, one cell (27 images)"))
    x, box, rl = _band_case()
    out.append((x, box, rl, "cutoff band, 3^3 cells"))
    return out


def test_static_pairs_equal_oracle_consecutive_calls():
    torch = pytest.importorskip("torch")
    from paper_2201_01446_gb300 import dp
    for rep in range(2):  # every case twice in a row through the shared scratch
        for x, box, rlist, tag in _cases():
            ref = oracle.neighbors(x, box, rlist, method=0 if len(x) < 600 else 1)
            got = dp.dp_neighbor_pairs_static(torch.tensor(x, device="cuda"), box, rlist)
            torch.cuda.synchronize()
            got = _sorted(got.cpu().numpy())
            assert got.shape == ref.shape and len(ref) > 0, tag
            assert np.array_equal(got, ref), tag


def test_static_pairs_equal_allocating_entry_point(cu_model_path):
    torch = pytest.importorskip("torch")
    from paper_2201_01446_gb300 import dp
    h = dp.dp_create(cu_model_path, 1, 8.0, 0.5, [256], stream=None)
    try:
        for x, box, rlist, tag in _cases():
            ref = _sorted(dp.dp_neighbor_pairs(h, x, box, rlist))
            got = dp.dp_neighbor_pairs_static(torch.tensor(x, device="cuda"), box, rlist)
            torch.cuda.synchronize()
            assert np.array_equal(_sorted(got.cpu().numpy()), ref), tag
    finally:
        dp.dp_destroy(h)


def test_static_pairs_capacity_below_count():
    # cap < count: the first cap rows of the library's order (atoms in index
    # order, each atom's rows in a fixed order) are written, nothing past them
    torch = pytest.importorskip("torch")
    from paper_2201_01446_gb300 import dp
    x, box, rlist, _ = _cases()[0]
    xt = torch.tensor(x, device="cuda")
    full = dp.dp_neighbor_pairs_static(xt, box, rlist).cpu().numpy()
    cap = len(full) // 3
    big = torch.full((cap + 64, 5), -7, dtype=torch.int32, device="cuda")
    _, cnt = dp.dp_neighbor_pairs_static(xt, box, rlist, out=big[:cap])
    torch.cuda.synchronize()
    b = big.cpu().numpy()
    assert cnt == len(full)
    assert np.array_equal(b[:cap], full[:cap])
    assert np.all(b[cap:] == -7)
    # cap = 0: the count alone
    _, cnt0 = dp.dp_neighbor_pairs_static(xt, box, rlist, out=big[:0])
    assert cnt0 == len(full)


def test_static_pairs_count_past_int32():
    # a simple cubic lattice of 32^3 sites in a box of edge rlist = 8 A
    # (spacing 0.25 A, exact in binary): every atom pairs with the sites k
    # (in lattice units, over all 27 images) with 0 < |k|^2 < 32^2, so the
    # total is N times that count, about 4.5e9, past any 32-bit offset
    torch = pytest.importorskip("torch")
    from paper_2201_01446_gb300 import dp
    n, L = 32, 8.0
    g = np.arange(n) * (L / n)
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    k = np.arange(-n + 1, n)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    per_atom = int(np.count_nonzero(k2 < n * n)) - 1
    expect = len(x) * per_atom
    assert expect > 2 ** 31
    xt = torch.tensor(x, device="cuda")
    box = np.diag([L, L, L])
    out = torch.full((4096, 5), -7, dtype=torch.int32, device="cuda")
    _, cnt = dp.dp_neighbor_pairs_static(xt, box, L, out=out)
    torch.cuda.synchronize()
    assert cnt == expect
    rows = out.cpu().numpy()
    # the first rows are atom 0's: distinct (j, image), each closer than rlist
    assert np.all(rows[:, 0] == 0)
    assert len(np.unique(rows[:, 1:], axis=0)) == len(rows)
    d = x[rows[:, 1]] + rows[:, 2:5] * L - x[0]
    assert np.all((d ** 2).sum(1) < L * L)


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
    # an edge / rlist ratio past any int: rejected, not converted
    with pytest.raises(dp.DPError) as e:
        dp.dp_neighbor_pairs_static(y, np.diag([1e12, 1e12, 1e12]), 1e-3)
    assert e.value.code == 12
