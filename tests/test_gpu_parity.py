"""CUDA path vs the FP64 oracle, element by element, through the C-ABI.

Bars:
  * neighbor sets bit-exact (as sorted (i, j, image) rows);
  * configured models (weights N(0, 0.1)): energy within 1e-6 eV/atom
    (|dE|/N), force RMSE within 1e-5 eV/A -- the FP32 path's stated
    tolerance -- and within 1e-3 of the reference RMS force (these models
    exert only ~1e-6 eV/A, so F = 0 must fail too), per-atom energies within
    1e-6 eV;
  * stress models (weights N(0, 1)): forces of 0.2-4 eV/A and per-atom
    energies of 7-40 eV, where FP32 rounding of the 2048-wide fitting net is
    ~1e-6 relative and does not average out over a near-perfect lattice.
    Their bars are relative: |dE|/N <= max(1e-6, 2e-6 mean|E_i|) eV,
    per-atom |dE_i| <= 2e-5 max|E_i|, force RMSE <= max(1e-5, 3e-5 RMS(F)),
    virial <= 1e-4 max|V|.
"""
import numpy as np
import pytest

import oracle
from paper_2201_01446_gb300 import inputs
from conftest import CU_RC, CU_RCS, CU_SEL, CU_SMAX, F_ABS, PARITY_LOG, TABLE_H, force_bar, rmse

pytestmark = pytest.mark.gpu

E_TOL = 1e-6   # eV/atom


@pytest.fixture(scope="module")
def dp():
    from paper_2201_01446_gb300 import dp as _dp
    return _dp


def _handle(dp, path, ntypes=1, rc=CU_RC, rcs=CU_RCS, sel=(CU_SEL,), **opt):
    o = dp.dp_options_default()
    for k, v in opt.items():
        setattr(o, k, v)
    return dp.dp_create(path, ntypes, rc, rcs, list(sel), options=o, stream=None)


@pytest.fixture(scope="module")
def cu(dp, cu_model_path):
    h = _handle(dp, cu_model_path)
    m = oracle.Model(cu_model_path)
    yield h, m, oracle.Table(m, TABLE_H, CU_SMAX)
    dp.dp_destroy(h)


@pytest.fixture(scope="module")
def cu_stress(dp, cu_stress_path):
    h = _handle(dp, cu_stress_path)
    m = oracle.Model(cu_stress_path)
    yield h, m, oracle.Table(m, TABLE_H, CU_SMAX)
    dp.dp_destroy(h)


def _sorted_rows(a):
    return a[np.lexsort(a.T[::-1])]


# ------------------------------------------------------------------ a1
@pytest.mark.parametrize("ncell,sigma,rlist", [(5, 0.05, 8.0), (5, 0.05, 10.0), (3, 0.3, 8.0),
                                               ((4, 3, 6), 0.2, 9.0), (9, 0.1, 10.0)])
def test_neighbor_sets_bit_exact(dp, cu, ncell, sigma, rlist):
    h, _, _ = cu
    x, _, box = inputs.fcc_copper(ncell, sigma=sigma, seed=21)
    x = x + np.array([-3.1, 17.0, 0.25])  # unwrapped input
    ref = oracle.neighbors(x, box, rlist, method=0 if len(x) < 600 else 1)
    got = _sorted_rows(dp.dp_neighbor_pairs(h, x, box, rlist))
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)


def test_neighbor_boundary_band(dp, cu):
    # pairs placed within 1e-7 A of the cutoff: the FP64 recheck decides
    h, _, _ = cu
    box = np.diag([30.0, 30.0, 30.0])
    rng = np.random.default_rng(5)
    xs = [np.array([15.0, 15.0, 15.0])]
    for k in range(40):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        xs.append(xs[0] + d * (8.0 + rng.choice([-1, 1]) * rng.uniform(0, 1e-7)))
    x = np.array(xs)
    ref = oracle.neighbors(x, box, 8.0, method=0)
    got = _sorted_rows(dp.dp_neighbor_pairs(h, x, box, 8.0))
    assert np.array_equal(got, ref)


# ------------------------------------------------------------------ table
def test_table_matches_oracle(dp, cu_stress):
    h, m, tab = cu_stress
    got = dp.dp_table_coeffs(h, 0, 0, M=m.M).astype(np.float64)
    ref = tab.coeffs(0, 0) * (TABLE_H ** np.arange(6))[None, :, None]
    assert got.shape == ref.shape
    scale = np.abs(ref).max(axis=1, keepdims=True) + 1e-30
    assert np.abs(got - ref).max() / scale.max() < 1e-6
    assert (np.abs(got - ref) / scale).max() < 1e-5


# ------------------------------------------------------------------ a2 + a3
def test_descriptor_matches_oracle(dp, cu_stress):
    h, m, tab = cu_stress
    x, t, box = inputs.fcc_copper(5, sigma=0.05, seed=1)
    T = dp.dp_descriptor(h, x, t, box, m.M)
    for i in [0, 17, 250, 499]:
        Tref, _ = oracle.atom_descriptor(m, tab, CU_RC, CU_RCS, CU_SEL, x, t, box, i)
        err = np.abs(T[i] - Tref).max()
        assert err < 2e-6 * np.abs(Tref).max(), (i, err)


# ------------------------------------------------------------------ a1..a9
def _parity(dp, h, m, tab, x, t, box, sel=CU_SEL, rc=CU_RC, rcs=CU_RCS, stress=False, tag="",
            e_rel=2e-6):
    E, F, V, Ei = dp.dp_compute(h, x, t, box, atom_energy=True)
    r = oracle.evaluate(m, tab, rc, rcs, sel, x, t, box)
    n = len(x)
    de = abs(E - r["energy"]) / n
    dei = float(np.abs(Ei - r["atom_energy"]).max()) if n else 0.0
    fr = rmse(F, r["force"])
    frms = float(np.sqrt((r["force"] ** 2).mean())) if n else 0.0
    dv = float(np.abs(V - r["virial"]).max())
    vmax = float(np.abs(r["virial"]).max())
    PARITY_LOG.append(dict(case=tag, natoms=n, stress=stress, dE_per_atom=de, max_dEi=dei,
                           force_rmse=fr, force_rms=frms, max_dvirial=dv, max_virial=vmax))
    if not stress:
        assert de < E_TOL, de
        assert dei < E_TOL, dei
        assert fr <= force_bar(frms), (fr, frms)
        assert dv < 1e-4 * max(vmax, 1e-3), (dv, vmax)
    else:
        emean = float(np.abs(r["atom_energy"]).mean())
        emax = float(np.abs(r["atom_energy"]).max())
        assert de < max(E_TOL, e_rel * emean), (de, emean)
        assert dei < 2e-5 * emax, (dei, emax)
        assert fr < max(F_ABS, 3e-5 * frms), (fr, frms)
        assert dv < 1e-4 * vmax + 1e-9, (dv, vmax)
    return E, F, V, r


def test_config1_parity(dp, cu):
    h, m, tab = cu
    x, t, box = inputs.fcc_copper(5, sigma=0.05, seed=1)
    _parity(dp, h, m, tab, x, t, box, tag="config1 Cu 500")


@pytest.mark.parametrize("ncell,sigma", [(5, 0.05), (3, 0.1), ((3, 4, 5), 0.15), (7, 0.1)])
def test_stress_parity(dp, cu_stress, ncell, sigma):
    h, m, tab = cu_stress
    x, t, box = inputs.fcc_copper(ncell, sigma=sigma, seed=2)
    _parity(dp, h, m, tab, x, t, box, stress=True, tag=f"stress Cu {ncell} {sigma}")


def test_ragged_random_positions(dp, cu_stress):
    # an irregular, non-lattice system: 333 atoms of a random packing
    h, m, tab = cu_stress
    rng = np.random.default_rng(8)
    L = 17.3
    pts = []
    while len(pts) < 333:
        p = rng.uniform(0, L, 3)
        if all(np.linalg.norm((p - q) - L * np.round((p - q) / L)) > 2.0 for q in pts):
            pts.append(p)
    x = np.array(pts)
    box = np.diag([L, L, L])
    _parity(dp, h, m, tab, x, np.zeros(len(x), np.int32), box, stress=True, tag="stress random 333")


@pytest.mark.parametrize("std", [0.1, 1.0])
def test_water_two_types(dp, model_dir, std):
    path = str(model_dir / f"water_std{std}.model")
    inputs.write_seeded_model(path, inputs.WATER_SPEC, seed=4, std=std)
    m = oracle.Model(path)
    tab = oracle.Table(m, TABLE_H, 1.25)
    h = _handle(dp, path, ntypes=2, rc=6.0, rcs=0.5, sel=(46, 92), s_max=1.25)
    try:
        x, t, box = inputs.water_like(64, L=12.417, seed=3)
        _parity(dp, h, m, tab, x, t, box, sel=[46, 92], rc=6.0, rcs=0.5, stress=std > 0.5,
                tag=f"water 192 std {std}")
    finally:
        dp.dp_destroy(h)


# ------------------------------------------------------------------ edge cases
def test_edge_cases(dp, cu_stress):
    h, m, tab = cu_stress
    box = np.diag([40.0, 40.0, 40.0])
    # empty system
    E, F, V, _ = dp.dp_compute(h, np.zeros((0, 3)), np.zeros(0, np.int32), box)
    assert E == 0.0 and F.shape == (0, 3) and np.all(V == 0)
    # one atom: no neighbors, E = fitting net at D = 0, F = 0
    E, F, V, _ = dp.dp_compute(h, np.array([[1.0, 2.0, 3.0]]), np.zeros(1, np.int32), box)
    E0, _ = m.fit(0, np.zeros(m.din))
    assert abs(E - E0) < 1e-5 and np.all(F == 0)
    # dimer and trimer
    for xs in ([[10, 10, 10], [12.5, 10.3, 9.8]], [[10, 10, 10], [12.5, 10.3, 9.8], [11, 12, 10.5]]):
        x = np.array(xs, float)
        _parity(dp, h, m, tab, x, np.zeros(len(x), np.int32), box, stress=True,
                tag=f"stress {len(x)} atoms")


def test_close_contacts(dp, cu_stress):
    # pairs at 1.2-1.6 A: s up to 0.8, far into the table, few members per interval
    h, m, tab = cu_stress
    x, t, box = inputs.fcc_copper(3, sigma=0.05, seed=9)
    x[1] = x[0] + np.array([1.2, 0.1, 0.0])
    x[7] = x[5] + np.array([0.2, 1.6, 0.3])
    _parity(dp, h, m, tab, x, t, box, stress=True, tag="close contacts")


def test_error_statuses(dp, cu_stress):
    h, m, tab = cu_stress
    x, t, box = inputs.fcc_copper(3, sigma=0.0)
    with pytest.raises(dp.DPError) as e:  # box edge 7.27 < rc
        xs, ts, bs = inputs.fcc_copper(2)
        dp.dp_compute(h, xs, ts, bs)
    assert e.value.code == 7
    skew = box.copy()
    skew[0, 1] = 0.5
    with pytest.raises(dp.DPError) as e:
        dp.dp_compute(h, x, t, skew)
    assert e.value.code == 7
    x2 = x.copy()
    x2[1] = x2[0] + np.array([0.45, 0, 0])  # s = 1/0.45 > 2
    with pytest.raises(dp.DPError) as e:
        dp.dp_compute(h, x2, t, box)
    assert e.value.code == 6
    with pytest.raises(dp.DPError) as e:
        dp.dp_compute(h, x, np.full(len(x), 3, np.int32), box)
    assert e.value.code == 1
    # the handle is still usable after errors
    xs, ts, bs = inputs.fcc_copper(3, sigma=0.1, seed=3)
    _parity(dp, h, m, tab, xs, ts, bs, stress=True, tag="after errors")


def test_sel_overflow(dp, cu_stress_path):
    h = _handle(dp, cu_stress_path, sel=(100,))
    try:
        x, t, box = inputs.fcc_copper(4, sigma=0.0)
        with pytest.raises(dp.DPError) as e:
            dp.dp_compute(h, x, t, box)
        assert e.value.code == 5
    finally:
        dp.dp_destroy(h)


@pytest.mark.parametrize("embed", [0, 2])
def test_sel_sections_at_their_limits_water(dp, water_model_path, embed):
    # N_m sectioned by neighbor type: with each section exactly at the largest
    # count of its type (counted here by a minimum-image brute force, rc = 6 <
    # L / 2) the evaluation runs and matches the oracle with the same sections
    # (which set N_m); one below in either section is DP_ERR_SEL_OVERFLOW
    m = oracle.Model(water_model_path)
    tab = oracle.Table(m, TABLE_H, 1.25)
    x, t, box = inputs.water_like(64, L=12.417, seed=3)
    L = np.diag(box)
    d = x[None, :, :] - x[:, None, :]
    d -= L * np.round(d / L)
    r2 = (d ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    within = r2 < 6.0 ** 2
    mx = [int((within & (t[None, :] == k)).sum(1).max()) for k in (0, 1)]
    for sel, ok in [(mx, True), ([mx[0] - 1, 92], False), ([46, mx[1] - 1], False)]:
        h = _handle(dp, water_model_path, ntypes=2, rc=6.0, rcs=0.5, sel=tuple(sel), s_max=1.25,
                    embed_precision=embed, fit_precision=0)
        try:
            if ok:
                # (the tensor-core contraction: the water allowance of its
                # total-energy accumulation bias, as in the other water cases)
                _parity(dp, h, m, tab, x, t, box, sel=sel, rc=6.0, rcs=0.5, stress=True,
                        tag=f"water sel at the counts {sel} embed {embed}",
                        e_rel=1e-5 if embed == 2 else 2e-6)
            else:
                with pytest.raises(dp.DPError) as e:
                    dp.dp_compute(h, x, t, box)
                assert e.value.code == 5, sel
        finally:
            dp.dp_destroy(h)


def test_bitwise_reproducible(dp, cu_stress):
    h, _, _ = cu_stress
    x, t, box = inputs.fcc_copper(6, sigma=0.1, seed=4)
    a = dp.dp_compute(h, x, t, box, atom_energy=True)
    b = dp.dp_compute(h, x, t, box, atom_energy=True)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert np.array_equal(a[3], b[3])


def test_device_pointer_path(dp, cu_stress):
    torch = pytest.importorskip("torch")
    h, m, tab = cu_stress
    x, t, box = inputs.fcc_copper(4, sigma=0.1, seed=6)
    E, F, V, Ei = dp.dp_compute(h, torch.tensor(x, device="cuda"),
                                torch.tensor(t, device="cuda"), torch.tensor(box, device="cuda"),
                                atom_energy=True)
    torch.cuda.synchronize()
    Eh, Fh, Vh, Eih = dp.dp_compute(h, x, t, box, atom_energy=True)
    assert float(E.cpu()[0]) == Eh
    assert np.array_equal(F.cpu().numpy(), Fh) and np.array_equal(V.cpu().numpy(), Vh)


# ------------------------------------------------------------------ plain untabulated path
@pytest.mark.parametrize("which", ["configured", "stress"])
def test_plain_untabulated_parity(dp, cu_model_path, cu_stress_path, which):
    # the comparator path evaluates the embedding net itself: compared with
    # the oracle's untabulated model (table = None)
    path = cu_model_path if which == "configured" else cu_stress_path
    m = oracle.Model(path)
    h = _handle(dp, path, tabulated=0)
    try:
        x, t, box = inputs.fcc_copper(5, sigma=0.05, seed=1)
        _parity(dp, h, m, None, x, t, box, stress=which == "stress", tag=f"plain Cu 500 {which}")
        xr, tr, br = inputs.fcc_copper((3, 4, 5), sigma=0.15, seed=2)
        _parity(dp, h, m, None, xr, tr, br, stress=which == "stress", tag=f"plain Cu 240 {which}")
    finally:
        dp.dp_destroy(h)


def test_plain_water_two_types(dp, water_model_path):
    m = oracle.Model(water_model_path)
    h = _handle(dp, water_model_path, ntypes=2, rc=6.0, rcs=0.5, sel=(46, 92), s_max=1.25,
                tabulated=0)
    try:
        x, t, box = inputs.water_like(64, L=12.417, seed=3)
        _parity(dp, h, m, None, x, t, box, sel=[46, 92], rc=6.0, rcs=0.5, stress=True,
                tag="plain water 192 std 1.0")
    finally:
        dp.dp_destroy(h)
