"""Pins of the oracle's parameter gradients (dE/d fitting weights and biases,
dE/d table coefficients, dE/d embedding-net weights and biases of the
original model) to central differences of the oracle's energy, to the exact
bias gradient and to the table's homogeneity (T is linear in the
coefficients, so sum_c c dE/dc = d/dlambda E(lambda c) at lambda = 1)."""
import numpy as np
import pytest

import oracle
from paper_2201_01446_gb300 import inputs

RC, RCS, SEL = 3.2, 0.5, [12, 24]
SPEC = inputs.ModelSpec(2, (8, 16, 32), 4, (24, 24, 24))


@pytest.fixture(scope="module")
def small(tmp_path_factory):
    path = str(tmp_path_factory.mktemp("pg") / "small.model")
    inputs.write_seeded_model(path, SPEC, seed=3, std=1.0)
    m = oracle.Model(path)
    tab = oracle.Table(m, 0.01, 1.25)
    x, t, box = inputs.water_like(8, L=6.5, seed=3)
    return m, tab, x, t, box


def _energy(m, tab, x, t, box):
    return oracle.evaluate(m, tab, RC, RCS, SEL, x, t, box)["energy"]


def test_energy_and_bias_gradient(small):
    m, tab, x, t, box = small
    E, gf, gt = oracle.param_grad(m, tab, RC, RCS, SEL, x, t, box)
    assert E == _energy(m, tab, x, t, box)
    # E = sum_i (z_i . w + b_out[t_i]): dE/db_out of type t is its atom count
    for ti in range(m.ntypes):
        assert gf[ti, -1] == float(np.sum(t == ti))
    assert gt.shape == (2, 2, tab.n, 6, m.M)


@pytest.mark.parametrize("ti", [0, 1])
def test_fitting_gradient_matches_central_differences(small, ti):
    m, tab, x, t, box = small
    _, gf, _ = oracle.param_grad(m, tab, RC, RCS, SEL, x, t, box)
    p0 = m.fit_params(ti)
    rng = np.random.default_rng(ti)
    # a sample over every block (first-layer W and b, hidden W and b, w_out)
    idx = list(rng.choice(len(p0), 12, replace=False)) + [0, len(p0) - 2, len(p0) - 30]
    try:
        for k in idx:
            eps = 1e-5 * max(1.0, abs(p0[k]))
            p = p0.copy()
            p[k] += eps
            m.set_fit_params(ti, p)
            ep = _energy(m, tab, x, t, box)
            p[k] -= 2 * eps
            m.set_fit_params(ti, p)
            em = _energy(m, tab, x, t, box)
            fd = (ep - em) / (2 * eps)
            assert abs(fd - gf[ti, k]) < 1e-7 + 1e-6 * abs(fd), (k, fd, gf[ti, k])
    finally:
        m.set_fit_params(ti, p0)


def test_table_gradient_matches_central_differences(small):
    m, tab, x, t, box = small
    _, _, gt = oracle.param_grad(m, tab, RC, RCS, SEL, x, t, box)
    h = tab.h
    big = np.argwhere(np.abs(gt) > 1e-3 * np.abs(gt).max())
    rng = np.random.default_rng(1)
    for k in rng.choice(len(big), 12, replace=False):
        ti, tj, kk, q, a = (int(v) for v in big[k])
        c0 = tab.coeffs(ti, tj)
        # the gradient is with respect to c_q = a_q h^q (the normalised local
        # variable); the oracle's table stores a_q
        eps = 1e-4
        try:
            c = c0.copy()
            c[kk, q, a] += eps / h ** q
            tab.set_coeffs(ti, tj, c)
            ep = _energy(m, tab, x, t, box)
            c[kk, q, a] -= 2 * eps / h ** q
            tab.set_coeffs(ti, tj, c)
            em = _energy(m, tab, x, t, box)
        finally:
            tab.set_coeffs(ti, tj, c0)
        fd = (ep - em) / (2 * eps)
        assert abs(fd - gt[ti, tj, kk, q, a]) < 1e-9 + 1e-6 * abs(fd), ((ti, tj, kk, q, a), fd)


def test_table_gradient_homogeneity(small):
    # T is linear in the coefficients: E(lambda c) has derivative sum c . dE/dc
    m, tab, x, t, box = small
    _, _, gt = oracle.param_grad(m, tab, RC, RCS, SEL, x, t, box)
    h = tab.h
    hq = h ** np.arange(6)
    lhs = 0.0
    c0 = [[tab.coeffs(a, b) for b in range(2)] for a in range(2)]
    for a in range(2):
        for b in range(2):
            lhs += float(np.sum(c0[a][b] * hq[None, :, None] * gt[a, b]))
    eps = 1e-5
    es = []
    try:
        for lam in (1 + eps, 1 - eps):
            for a in range(2):
                for b in range(2):
                    tab.set_coeffs(a, b, c0[a][b] * lam)
            es.append(_energy(m, tab, x, t, box))
    finally:
        for a in range(2):
            for b in range(2):
                tab.set_coeffs(a, b, c0[a][b])
    fd = (es[0] - es[1]) / (2 * eps)
    assert abs(fd - lhs) < 1e-6 * max(1.0, abs(fd)), (fd, lhs)


def test_untabulated_fitting_gradient(small):
    # the original embedding net: fitting gradients only, same central-difference pin
    m, _, x, t, box = small
    E, gf, gt = oracle.param_grad(m, None, RC, RCS, SEL, x, t, box, with_table=False)
    assert gt is None and E == _energy(m, None, x, t, box)
    p0 = m.fit_params(1)
    k = len(p0) // 3
    eps = 1e-5
    try:
        p = p0.copy()
        p[k] += eps
        m.set_fit_params(1, p)
        ep = _energy(m, None, x, t, box)
        p[k] -= 2 * eps
        m.set_fit_params(1, p)
        em = _energy(m, None, x, t, box)
    finally:
        m.set_fit_params(1, p0)
    assert abs((ep - em) / (2 * eps) - gf[1, k]) < 1e-7 + 1e-6 * abs(gf[1, k])


@pytest.mark.parametrize("pair", [(0, 0), (0, 1), (1, 1)])
def test_embedding_net_gradient_matches_central_differences(small, pair):
    # the original (untabulated) model: dE/d(embedding-net weights, biases)
    m, _, x, t, box = small
    ti, tj = pair
    _, _, ge = oracle.param_grad(m, None, RC, RCS, SEL, x, t, box)
    assert ge.shape == (2, 2, m.n_emb_params)
    p0 = m.emb_params(ti, tj)
    rng = np.random.default_rng(3 + ti + 2 * tj)
    # W_0, b_0, a hidden W and b, the last layer's W and b
    idx = [0, 9, 20] + list(rng.choice(len(p0), 9, replace=False)) + [len(p0) - 1]
    try:
        for k in idx:
            eps = 1e-5 * max(1.0, abs(p0[k]))
            p = p0.copy()
            p[k] += eps
            m.set_emb_params(ti, tj, p)
            ep = _energy(m, None, x, t, box)
            p[k] -= 2 * eps
            m.set_emb_params(ti, tj, p)
            em = _energy(m, None, x, t, box)
            fd = (ep - em) / (2 * eps)
            assert abs(fd - ge[ti, tj, k]) < 1e-8 + 1e-6 * abs(fd), (k, fd, ge[ti, tj, k])
    finally:
        m.set_emb_params(ti, tj, p0)


def test_table_gradient_with_extrapolation_region(small):
    # coarse intervals (width H = 10 h beyond s = 0.4): the gradient is with
    # respect to c_q = a_q w^q, w the interval's own width
    m, _, x, t, box = small
    tab = oracle.Table(m, 0.01, 0.4, s_ext=1.25, ext_stride=10)
    assert tab.n_fine == 40 and tab.n == 49
    _, _, gt = oracle.param_grad(m, tab, RC, RCS, SEL, x, t, box)
    w = tab.widths()
    big = np.argwhere(np.abs(gt) > 1e-3 * np.abs(gt).max())
    coarse = big[big[:, 2] >= tab.n_fine]
    fine = big[big[:, 2] < tab.n_fine]
    assert len(coarse) >= 6 and len(fine) >= 6
    rng = np.random.default_rng(2)
    picks = list(coarse[rng.choice(len(coarse), 6, replace=False)]) + \
        list(fine[rng.choice(len(fine), 3, replace=False)])
    for ti, tj, kk, q, a in (tuple(int(v) for v in p) for p in picks):
        c0 = tab.coeffs(ti, tj)
        eps = 1e-4
        try:
            c = c0.copy()
            c[kk, q, a] += eps / w[kk] ** q
            tab.set_coeffs(ti, tj, c)
            ep = _energy(m, tab, x, t, box)
            c[kk, q, a] -= 2 * eps / w[kk] ** q
            tab.set_coeffs(ti, tj, c)
            em = _energy(m, tab, x, t, box)
        finally:
            tab.set_coeffs(ti, tj, c0)
        fd = (ep - em) / (2 * eps)
        assert abs(fd - gt[ti, tj, kk, q, a]) < 1e-9 + 1e-6 * abs(fd), ((ti, tj, kk, q, a), fd)
