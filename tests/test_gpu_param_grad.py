"""Parameter gradients through the C-ABI (dp_param_grad) against the FP64
oracle's: dE/d(fitting weights and biases) and dE/d(table coefficients), on
the configured copper model (500 atoms: 15 full tiles and a ragged one) and
the two-type water model (four type-pair tables, two fitting nets), plus the
exact output-bias gradient, determinism and the degenerate cases."""
import numpy as np
import pytest

import oracle
from paper_2201_01446_gb300 import inputs
from conftest import CU_RC, CU_RCS, CU_SEL, CU_SMAX, PARITY_LOG, TABLE_H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    from paper_2201_01446_gb300 import dp as _dp
    return _dp


def _blocks(spec_din, widths):
    """(name, start, shape) of one type's fitting-gradient layout."""
    out, o, win = [], 0, spec_din
    for k, w in enumerate(widths):
        out.append((f"W{k}", o, (win, w)))
        o += win * w
        out.append((f"b{k}", o, (w,)))
        o += w
        win = w
    out.append(("w_out", o, (win,)))
    out.append(("b_out", o + win, (1,)))
    return out


def _compare_fit(g_gpu, g_orc, m, widths, tag, bar):
    per = m.n_fit_params
    worst = {}
    for ti in range(m.ntypes):
        for name, o, shape in _blocks(m.din, widths):
            n = int(np.prod(shape))
            a = g_gpu[ti * per + o: ti * per + o + n]
            b = g_orc[ti, o: o + n]
            scale = float(np.abs(b).max())
            err = float(np.abs(a - b).max())
            worst[f"t{ti} {name}"] = err / max(scale, 1e-300)
            assert err <= bar * scale + 1e-12, (tag, ti, name, err, scale)
    return worst


def _node_intervals(x, t, box, rc, rcs, h):
    """(ti, tj, k) of the intervals next to a table node that some pair's s
    lies within 1e-4 h of: FP32 and FP64 may put such a pair on different
    sides of the node, and the coefficient gradient (unlike the energy) jumps
    there, so these intervals are left out of the elementwise comparison."""
    out = set()
    for i, j, n0, n1, n2 in oracle.neighbors(x, box, rc):
        d = x[j] + np.array([n0, n1, n2]) * np.diag(box) - x[i]
        s, _, _ = oracle.env_row(d, rc, rcs)
        q = s / h
        k = int(round(q))
        if abs(q - k) < 1e-4:
            out.update({(int(t[i]), int(t[j]), k - 1), (int(t[i]), int(t[j]), k)})
    return out


def _compare_table(g_gpu, g_orc, tag, bar, skip=()):
    g_gpu = g_gpu.reshape(g_orc.shape).copy()
    g_orc = g_orc.copy()
    for a, b, k in skip:
        if 0 <= k < g_orc.shape[2]:
            g_gpu[a, b, k] = g_orc[a, b, k] = 0.0
    rel = {}
    for a in range(g_orc.shape[0]):
        for b in range(g_orc.shape[1]):
            x, y = g_gpu[a, b], g_orc[a, b]
            scale = float(np.abs(y).max())
            err = float(np.abs(x - y).max())
            rel[f"{a}{b}"] = err / max(scale, 1e-300)
            assert err <= bar * scale + 1e-12, (tag, a, b, err, scale)
            # intervals no pair visits stay exactly zero
            assert not x[y == 0.0].any(), (tag, a, b)
    return rel


def _handle(dp, path, ntypes, rc, rcs, sel, s_max):
    o = dp.dp_options_default()
    o.embed_precision = 2
    o.s_max = s_max
    return dp.dp_create(path, ntypes, rc, rcs, list(sel), options=o, stream=None)


def test_param_grad_copper(dp, cu_stress_path):
    m = oracle.Model(cu_stress_path)
    tab = oracle.Table(m, TABLE_H, CU_SMAX)
    x, t, box = inputs.fcc_copper(5, sigma=0.05, seed=1)
    E0, gf0, gt0 = oracle.param_grad(m, tab, CU_RC, CU_RCS, CU_SEL, x, t, box)
    h = _handle(dp, cu_stress_path, 1, CU_RC, CU_RCS, (CU_SEL,), CU_SMAX)
    try:
        E, gf, gt = dp.dp_param_grad(h, x, t, box)
        E2, gf2, gt2 = dp.dp_param_grad(h, x, t, box)
    finally:
        dp.dp_destroy(h)
    # deterministic: per-CTA partials and fixed-order reductions
    assert E == E2 and np.array_equal(gf, gf2) and np.array_equal(gt, gt2)
    assert gf[-1] == len(x)  # dE/db_out = number of atoms
    assert abs(E - E0) / len(x) < max(1e-6, 5e-6 * abs(E0) / len(x))
    skip = _node_intervals(x, t, box, CU_RC, CU_RCS, TABLE_H)
    wf = _compare_fit(gf, gf0, m, inputs.COPPER_SPEC.fit_w, "Cu", 2e-5)
    wt = _compare_table(gt, gt0, "Cu", 2e-5, skip)
    PARITY_LOG.append(dict(case="param grad Cu 500 std 1.0", natoms=len(x), dE=abs(E - E0),
                           fit_max_err_over_block_max=max(wf.values()),
                           table_max_err_over_max=max(wt.values()), node_intervals_skipped=len(skip)))


def test_param_grad_water_two_types(dp, water_model_path):
    m = oracle.Model(water_model_path)
    tab = oracle.Table(m, TABLE_H, 1.25)
    x, t, box = inputs.water_like(64, L=12.417, seed=3)
    E0, gf0, gt0 = oracle.param_grad(m, tab, 6.0, 0.5, [46, 92], x, t, box)
    h = _handle(dp, water_model_path, 2, 6.0, 0.5, (46, 92), 1.25)
    try:
        E, gf, gt = dp.dp_param_grad(h, x, t, box)
    finally:
        dp.dp_destroy(h)
    per = m.n_fit_params
    assert gf[per - 1] == 64 and gf[2 * per - 1] == 128
    skip = _node_intervals(x, t, box, 6.0, 0.5, TABLE_H)
    wf = _compare_fit(gf, gf0, m, inputs.WATER_SPEC.fit_w, "water", 2e-5)
    wt = _compare_table(gt, gt0, "water", 2e-5, skip)
    PARITY_LOG.append(dict(case="param grad water 192 std 1.0", natoms=len(x), dE=abs(E - E0),
                           fit_max_err_over_block_max=max(wf.values()),
                           table_max_err_over_max=max(wt.values()), node_intervals_skipped=len(skip)))


def test_param_grad_edge_cases(dp, cu_model_path):
    h = _handle(dp, cu_model_path, 1, CU_RC, CU_RCS, (CU_SEL,), CU_SMAX)
    try:
        box = np.diag([40.0, 40.0, 40.0])
        E, gf, gt = dp.dp_param_grad(h, np.zeros((0, 3)), np.zeros(0, np.int32), box)
        assert E == 0.0 and not gf.any() and not gt.any()
        # one isolated atom: D = 0, the net's gradient at zero input, no table use
        m = oracle.Model(cu_model_path)
        x1 = np.array([[1.0, 2.0, 3.0]])
        E, gf, gt = dp.dp_param_grad(h, x1, np.zeros(1, np.int32), box)
        E0, gf0, _ = oracle.param_grad(m, None, CU_RC, CU_RCS, CU_SEL, x1, np.zeros(1, np.int32),
                                       box)
        assert not gt.any() and gf[-1] == 1.0
        assert np.abs(gf - gf0[0]).max() < 1e-5 * np.abs(gf0).max()
    finally:
        dp.dp_destroy(h)
    # table gradients need the tensor-core embedding's sorted pairs
    o = dp.dp_options_default()
    o.embed_precision = 0
    h0 = dp.dp_create(cu_model_path, 1, CU_RC, CU_RCS, [CU_SEL], options=o, stream=None)
    try:
        x, t, bx = inputs.fcc_copper(3, sigma=0.05, seed=2)
        with pytest.raises(dp.DPError) as e:
            dp.dp_param_grad(h0, x, t, bx, table=True)
        assert e.value.code == 9
        E, gf, gt = dp.dp_param_grad(h0, x, t, bx, table=False)
        assert gt is None and gf[-1] == len(x)
    finally:
        dp.dp_destroy(h0)


def test_set_params_matches_oracle_and_autograd(dp, cu_stress_path):
    torch = pytest.importorskip("torch")
    from paper_2201_01446_gb300 import autograd
    m = oracle.Model(cu_stress_path)
    tab = oracle.Table(m, TABLE_H, CU_SMAX)
    x, t, box = inputs.fcc_copper(4, sigma=0.05, seed=5)
    h = _handle(dp, cu_stress_path, 1, CU_RC, CU_RCS, (CU_SEL,), CU_SMAX)
    try:
        fit0, tab0 = dp.dp_get_params(h)
        dp.dp_set_params(h, fit0, tab0)
        f1, t1 = dp.dp_get_params(h)
        assert np.array_equal(f1, fit0) and np.array_equal(t1, tab0)  # FP32 values round-trip
        # new parameters on both sides: scaled fitting weights, a reshaped table
        rng = np.random.default_rng(0)
        fit = fit0 * (1.0 + 0.05 * rng.standard_normal(fit0.size))
        table = tab0 * (1.0 + 0.02 * rng.standard_normal(tab0.size))
        dp.dp_set_params(h, fit, table)
        fit32, table32 = dp.dp_get_params(h)
        E, F, V, _ = dp.dp_compute(h, x, t, box)
        m.set_fit_params(0, fit32)
        n, M = tab.n, m.M
        tab.set_coeffs(0, 0, table32.reshape(n, 6, M) / TABLE_H ** np.arange(6)[None, :, None])
        r = oracle.evaluate(m, tab, CU_RC, CU_RCS, CU_SEL, x, t, box)
        frms = float(np.sqrt((r["force"] ** 2).mean()))
        assert abs(E - r["energy"]) / len(x) < max(1e-6, 2e-6 * float(np.abs(r["atom_energy"]).mean()))
        assert float(np.sqrt(((F - r["force"]) ** 2).mean())) < max(1e-5, 3e-5 * frms)
        # the energy as a torch function of the parameters
        pf = torch.tensor(fit32, requires_grad=True)
        pt = torch.tensor(table32, requires_grad=True)
        Et = autograd.energy_params(h, pf, pt, x, t, box)
        Et.backward()
        E2, gf, gt = dp.dp_param_grad(h, x, t, box)
        assert float(Et.detach()) == E2
        assert np.array_equal(pf.grad.numpy(), gf) and np.array_equal(pt.grad.numpy(), gt)
        # a gradient step on the fitting parameters lowers E by eta |g|^2 to
        # first order: E(p - eta g) = E - eta |g|^2 + O(eta^2); two step
        # sizes remove the second-order term (Richardson)
        g2 = float(gf @ gf)
        eta = 1e-3 * abs(E2) / g2
        ratios = []
        for step in (eta, eta / 2):
            E3 = float(autograd.energy_params(h, torch.tensor(fit32 - step * gf), None, x, t, box))
            ratios.append((E2 - E3) / (step * g2))
        r_ex = 2 * ratios[1] - ratios[0]
        PARITY_LOG.append(dict(case="param set + gradient step Cu 256", ratios=ratios,
                               extrapolated=r_ex))
        assert ratios[0] > 0 and abs(r_ex - 1.0) < 0.05, ratios
    finally:
        dp.dp_destroy(h)


def test_param_grad_tanh_table(dp, cu_stress_path):
    # the fitting net on the Sec. 3.5 tanh table: the gradients use the
    # table's own derivative on both sides
    m = oracle.Model(cu_stress_path)
    tab = oracle.Table(m, TABLE_H, CU_SMAX)
    x, t, box = inputs.fcc_copper(4, sigma=0.05, seed=8)
    oracle.set_tanh_table(True)
    try:
        E0, gf0, gt0 = oracle.param_grad(m, tab, CU_RC, CU_RCS, CU_SEL, x, t, box)
    finally:
        oracle.set_tanh_table(False)
    o = dp.dp_options_default()
    o.embed_precision = 2
    o.tanh_table = 1
    h = dp.dp_create(cu_stress_path, 1, CU_RC, CU_RCS, [CU_SEL], options=o, stream=None)
    try:
        E, gf, gt = dp.dp_param_grad(h, x, t, box)
    finally:
        dp.dp_destroy(h)
    skip = _node_intervals(x, t, box, CU_RC, CU_RCS, TABLE_H)
    wf = _compare_fit(gf, gf0, m, inputs.COPPER_SPEC.fit_w, "Cu tanh table", 2e-5)
    wt = _compare_table(gt, gt0, "Cu tanh table", 2e-5, skip)
    PARITY_LOG.append(dict(case="param grad Cu 256 tanh table", dE=abs(E - E0),
                           fit_max_err_over_block_max=max(wf.values()),
                           table_max_err_over_max=max(wt.values())))


def _emb_blocks(d1, M):
    d2 = 2 * d1
    return [("W0", 0, d1), ("b0", d1, d1), ("W1", 2 * d1, d1 * d2), ("b1", 2 * d1 + d1 * d2, d2),
            ("W2", 2 * d1 + d1 * d2 + d2, d2 * M), ("b2", 2 * d1 + d1 * d2 + d2 + d2 * M, M)]


@pytest.mark.parametrize("case", ["cu", "water"])
def test_param_grad_untabulated(dp, cu_stress_path, water_model_path, case):
    # the original embedding nets (tabulated = 0): dE/d(embedding weights and
    # biases) per type pair on the plain path, and the fitting gradients
    if case == "cu":
        path, nt, rc, rcs, sel, spec = cu_stress_path, 1, CU_RC, CU_RCS, [CU_SEL], inputs.COPPER_SPEC
        x, t, box = inputs.fcc_copper(4, sigma=0.05, seed=9)
    else:
        path, nt, rc, rcs, sel, spec = water_model_path, 2, 6.0, 0.5, [46, 92], inputs.WATER_SPEC
        x, t, box = inputs.water_like(64, L=12.417, seed=3)
    m = oracle.Model(path)
    E0, gf0, ge0 = oracle.param_grad(m, None, rc, rcs, sel, x, t, box)
    o = dp.dp_options_default()
    o.tabulated = 0
    h = dp.dp_create(path, nt, rc, rcs, sel, options=o, stream=None)
    try:
        E, gf, ge = dp.dp_param_grad(h, x, t, box)
        fit, emb = dp.dp_get_params(h)
    finally:
        dp.dp_destroy(h)
    npar = m.n_emb_params
    assert ge.size == nt * nt * npar
    # the handle's embedding parameters are the model's, in the same layout
    for a in range(nt):
        for b in range(nt):
            assert np.array_equal(emb[(a * nt + b) * npar:(a * nt + b + 1) * npar], m.emb_params(a, b))
    wf = _compare_fit(gf, gf0, m, spec.fit_w, f"{case} plain", 2e-5)
    worst = 0.0
    ge = ge.reshape(nt, nt, npar)
    for a in range(nt):
        for b in range(nt):
            for name, o0, cnt in _emb_blocks(spec.emb_w[0], spec.emb_w[-1]):
                u, v = ge[a, b, o0:o0 + cnt], ge0[a, b, o0:o0 + cnt]
                scale = float(np.abs(v).max())
                err = float(np.abs(u - v).max())
                worst = max(worst, err / max(scale, 1e-300))
                assert err <= 2e-5 * scale + 1e-12, (case, a, b, name, err, scale)
    PARITY_LOG.append(dict(case=f"param grad {case} untabulated", dE=abs(E - E0),
                           fit_max_err_over_block_max=max(wf.values()),
                           emb_max_err_over_block_max=worst))


def test_set_params_untabulated_embedding_nets(dp, water_model_path):
    # new embedding nets on an untabulated handle: energy and forces follow
    # the oracle's original model with the same nets; the handle returns
    # them as given; a torch step on them matches dp_param_grad
    torch = pytest.importorskip("torch")
    from paper_2201_01446_gb300 import autograd
    m = oracle.Model(water_model_path)
    x, t, box = inputs.water_like(64, L=12.417, seed=7)
    o = dp.dp_options_default()
    o.tabulated = 0
    h = dp.dp_create(water_model_path, 2, 6.0, 0.5, [46, 92], options=o, stream=None)
    npar = m.n_emb_params
    try:
        fit0, emb0 = dp.dp_get_params(h)
        rng = np.random.default_rng(4)
        emb = emb0 * (1.0 + 0.05 * rng.standard_normal(emb0.size))
        dp.dp_set_params(h, None, emb)
        _, emb1 = dp.dp_get_params(h)
        assert np.array_equal(emb1, emb)
        E, F, V, _ = dp.dp_compute(h, x, t, box)
        for a in range(2):
            for b in range(2):
                q = a * 2 + b
                m.set_emb_params(a, b, emb[q * npar:(q + 1) * npar])
        r = oracle.evaluate(m, None, 6.0, 0.5, [46, 92], x, t, box)
        frms = float(np.sqrt((r["force"] ** 2).mean()))
        assert abs(E - r["energy"]) / len(x) < max(1e-6, 2e-6 * float(np.abs(r["atom_energy"]).mean()))
        assert float(np.sqrt(((F - r["force"]) ** 2).mean())) < max(1e-5, 3e-5 * frms)
        assert np.abs(V - r["virial"]).max() < 1e-4 * np.abs(r["virial"]).max() + 1e-9
        # the energy as a torch function of the embedding nets
        pe = torch.tensor(emb, requires_grad=True)
        Et = autograd.energy_params(h, torch.tensor(fit0), pe, x, t, box)
        Et.backward()
        E2, _, ge = dp.dp_param_grad(h, x, t, box)
        assert float(Et.detach()) == E2 and np.array_equal(pe.grad.numpy(), ge)
        PARITY_LOG.append(dict(case="set embedding nets, water 192 untabulated",
                               dE_per_atom=abs(E - r["energy"]) / len(x)))
    finally:
        dp.dp_destroy(h)
