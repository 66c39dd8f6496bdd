"""The table's extrapolation region (dp_options.s_ext, ext_stride) against the
oracle's table with the same layout: intervals of width h up to s_max, then
of width ext_stride * h up to s_ext.  A fine region that ends at s = 0.3
puts copper's nearest neighbors (s ~ 0.34) into the coarse intervals, so
both regions are exercised.  Bars as in the parity tests (relative for the
stress model)."""
import numpy as np
import pytest

import oracle
from paper_2201_01446_gb300 import inputs
from conftest import CU_RC, CU_RCS, CU_SEL, PARITY_LOG, TABLE_H, rmse

pytestmark = pytest.mark.gpu

S_MAX, S_EXT, STRIDE = 0.3, 2.0, 10


@pytest.fixture(scope="module")
def dp():
    from paper_2201_01446_gb300 import dp as _dp
    return _dp


def _handle(dp, path, embed_precision, s_ext=S_EXT, ntypes=1, rc=CU_RC, rcs=CU_RCS,
            sel=(CU_SEL,), s_max=S_MAX):
    o = dp.dp_options_default()
    o.s_max = s_max
    o.s_ext = s_ext
    o.ext_stride = STRIDE
    o.embed_precision = embed_precision
    return dp.dp_create(path, ntypes, rc, rcs, list(sel), options=o, stream=None)


def test_table_layout_matches_oracle(dp, cu_stress_path):
    m = oracle.Model(cu_stress_path)
    tab = oracle.Table(m, TABLE_H, S_MAX, s_ext=S_EXT, ext_stride=STRIDE)
    h = _handle(dp, cu_stress_path, 0)
    try:
        got = dp.dp_table_coeffs(h, 0, 0, M=m.M).astype(np.float64)
    finally:
        dp.dp_destroy(h)
    assert got.shape[0] == tab.n == 30 + 17
    # the device stores the coefficients of u = (s - x_k) / w_k
    ref = tab.coeffs(0, 0) * tab.widths()[:, None, None] ** np.arange(6)[None, :, None]
    scale = np.abs(ref).max(axis=1, keepdims=True) + 1e-30
    assert (np.abs(got - ref) / scale).max() < 1e-5


@pytest.mark.parametrize("embed_precision", [0, 2])
@pytest.mark.parametrize("cells,sigma", [(5, 0.05), ((3, 4, 5), 0.15)])
def test_parity_with_extrapolation_region(dp, cu_stress_path, embed_precision, cells, sigma):
    m = oracle.Model(cu_stress_path)
    tab = oracle.Table(m, TABLE_H, S_MAX, s_ext=S_EXT, ext_stride=STRIDE)
    x, t, box = inputs.fcc_copper(cells, sigma=sigma, seed=4)
    h = _handle(dp, cu_stress_path, embed_precision)
    try:
        E, F, V, Ei = dp.dp_compute(h, x, t, box, atom_energy=True)
    finally:
        dp.dp_destroy(h)
    r = oracle.evaluate(m, tab, CU_RC, CU_RCS, CU_SEL, x, t, box)
    n = len(x)
    de = abs(E - r["energy"]) / n
    emean = float(np.abs(r["atom_energy"]).mean())
    emax = float(np.abs(r["atom_energy"]).max())
    frms = float(np.sqrt((r["force"] ** 2).mean()))
    fr = rmse(F, r["force"])
    dv = float(np.abs(V - r["virial"]).max())
    vmax = float(np.abs(r["virial"]).max())
    PARITY_LOG.append(dict(case=f"table extrapolation region, Cu {cells} {sigma}, "
                                f"embed_precision {embed_precision}", natoms=n,
                           dE_per_atom=de, force_rmse=fr, force_rms=frms))
    assert de < max(1e-6, 2e-6 * emean), (de, emean)
    assert float(np.abs(Ei - r["atom_energy"]).max()) < 2e-5 * emax
    assert fr < max(1e-5, 3e-5 * frms), (fr, frms)
    assert dv < 1e-4 * vmax + 1e-9, (dv, vmax)


def test_extrapolation_region_range_and_gradient(dp, cu_stress_path):
    # beyond the last node of the coarse region: DP_ERR_TABLE_RANGE; without
    # the region the same configuration is out of range of the fine table
    m = oracle.Model(cu_stress_path)
    x, t, box = inputs.fcc_copper(3, sigma=0.05, seed=5)
    h0 = _handle(dp, cu_stress_path, 2, s_ext=0.0)
    try:
        with pytest.raises(dp.DPError) as e:
            dp.dp_compute(h0, x, t, box)
        assert e.value.code == 6
    finally:
        dp.dp_destroy(h0)
    x2 = x.copy()
    x2[1] = x2[0] + np.array([0.45, 0.0, 0.0])  # s = 1/0.45 > 2.0 = s_ext
    h = _handle(dp, cu_stress_path, 2)
    try:
        with pytest.raises(dp.DPError) as e:
            dp.dp_compute(h, x2, t, box)
        assert e.value.code == 6
        # the table gradient with respect to each interval's normalised
        # coefficients matches the oracle's (same layout)
        E, gf, gt = dp.dp_param_grad(h, x, t, box)
    finally:
        dp.dp_destroy(h)
    tab = oracle.Table(m, TABLE_H, S_MAX, s_ext=S_EXT, ext_stride=STRIDE)
    E0, _, gt0 = oracle.param_grad(m, tab, CU_RC, CU_RCS, CU_SEL, x, t, box)
    gt = gt.reshape(gt0.shape).copy()
    gt0 = gt0.copy()
    # a pair whose s lies within 1e-4 of a width from a node may fall on
    # either side of it in FP32 and FP64: the coefficient gradient jumps
    # there, so the two intervals at such a node are left out
    nodes, widths = tab.nodes(), tab.widths()
    for i, j, n0, n1, n2 in oracle.neighbors(x, box, CU_RC):
        d = x[j] + np.array([n0, n1, n2]) * np.diag(box) - x[i]
        sv, _, _ = oracle.env_row(d, CU_RC, CU_RCS)
        k = int(np.argmin(np.abs(nodes - sv)))
        if abs(nodes[k] - sv) < 1e-4 * widths[min(k, tab.n - 1)]:
            for kk in (k - 1, k):
                if 0 <= kk < tab.n:
                    gt[0, 0, kk] = gt0[0, 0, kk] = 0.0
    assert np.abs(gt0[0, 0, tab.n_fine:]).max() > 0.0  # the coarse region is used
    err = np.abs(gt - gt0).max() / np.abs(gt0).max()
    assert not gt[gt0 == 0.0].any()  # intervals no pair visits stay zero
    PARITY_LOG.append(dict(case="table gradient with extrapolation region, Cu 108",
                           dE=abs(E - E0), table_max_err_over_max=float(err)))
    assert err < 2e-5, err
