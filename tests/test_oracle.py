"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's formulas: each checks a closed form, an
invariance, a derivative identity, an exactness property or a brute-force
count, chosen so that a dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2201_01446_gb300 import inputs
from conftest import CU_RC, CU_RCS, CU_SEL, CU_SMAX, TABLE_H, rmse

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- Eq. 1 gate
def test_switch_closed_form_properties():
    rc, rcs = 8.0, 0.5
    # sw = 1 inside rcs, 0 beyond rc, 1/2 at the midpoint (u -> 1-u symmetry)
    assert oracle.switch(0.3, rc, rcs) == (1.0, 0.0)
    assert oracle.switch(8.0, rc, rcs) == (0.0, 0.0)
    assert oracle.switch(9.0, rc, rcs) == (0.0, 0.0)
    assert abs(oracle.switch(0.5 * (rc + rcs), rc, rcs)[0] - 0.5) < 1e-15
    for u in [0.1, 0.27, 0.4]:
        a = oracle.switch(rcs + u * (rc - rcs), rc, rcs)[0]
        b = oracle.switch(rcs + (1 - u) * (rc - rcs), rc, rcs)[0]
        assert abs(a + b - 1.0) < 1e-14
    # C2 at both ends: value, slope and curvature continuous
    for r0, inside in [(rcs, 1.0), (rc, 0.0)]:
        for eps in [1e-4, 1e-3]:
            lo, dlo = oracle.switch(r0 - eps, rc, rcs)
            hi, dhi = oracle.switch(r0 + eps, rc, rcs)
            assert abs(lo - hi) < 50 * eps ** 3
            assert abs(dlo - dhi) < 50 * eps ** 2
    # derivative is the derivative
    h = 1e-6
    for r in np.linspace(0.6, 7.9, 17):
        fd = (oracle.switch(r + h, rc, rcs)[0] - oracle.switch(r - h, rc, rcs)[0]) / (2 * h)
        assert abs(fd - oracle.switch(r, rc, rcs)[1]) < 1e-8
    # monotone decreasing
    v = [oracle.switch(r, rc, rcs)[0] for r in np.linspace(0.5, 8.0, 200)]
    assert all(a >= b for a, b in zip(v, v[1:]))


def test_env_row_structure_and_derivative():
    rng = np.random.default_rng(0)
    rc, rcs = 6.0, 0.5
    for _ in range(20):
        d = rng.normal(size=3)
        d *= rng.uniform(0.7, 5.9) / np.linalg.norm(d)
        s, R, dR = oracle.env_row(d, rc, rcs)
        r = np.linalg.norm(d)
        sw, _ = oracle.switch(r, rc, rcs)
        assert abs(R[0] - sw / r) < 1e-15 and abs(s - R[0]) == 0
        # rows 1..3 are s times the unit vector: length s, direction d
        assert abs(np.linalg.norm(R[1:]) - R[0]) < 1e-14
        assert np.allclose(np.cross(R[1:], d), 0, atol=1e-14)
        # rotation covariance
        Q = inputs._random_rotation(rng)
        _, R2, _ = oracle.env_row(Q @ d, rc, rcs)
        assert abs(R2[0] - R[0]) < 1e-14 and np.allclose(R2[1:], Q @ R[1:], atol=1e-14)
        # Jacobian by central differences
        h = 1e-6
        for b in range(3):
            e = np.zeros(3)
            e[b] = h
            fd = (oracle.env_row(d + e, rc, rcs)[1] - oracle.env_row(d - e, rc, rcs)[1]) / (2 * h)
            assert np.allclose(fd, dR[:, b], atol=1e-8)


# ------------------------------------------------------------ Eq. 3-5 (embedding)
def _special_model(tmp_path, name, mutate, spec=inputs.COPPER_SPEC, seed=5, std=0.5):
    arrs = inputs.make_model(spec, seed, std)
    mutate(arrs)
    p = tmp_path / name
    inputs.write_model(p, spec, arrs)
    return oracle.Model(p), arrs


def test_embedding_reduces_to_closed_form(tmp_path):
    # zero W1, W2 and b2: layer 1 gives (h0,h0)+tanh(b1), layer 2 repeats it;
    # g[c] = tanh(s W0[c%32] + b0[c%32]) + tanh(b1[c%64]) pins the (x,x)
    # concatenation order of Eq. 5 and the tanh of Eq. 4
    def mut(a):
        a["emb00_W1"][:] = 0
        a["emb00_W2"][:] = 0
        a["emb00_b2"][:] = 0
    m, a = _special_model(tmp_path, "emb.model", mut)
    c = np.arange(128)
    for s in [0.0, 0.13, 0.4]:
        g, dg, d2g = m.embed(0, 0, s)
        z = s * a["emb00_W0"][c % 32] + a["emb00_b0"][c % 32]
        ref = np.tanh(z) + np.tanh(a["emb00_b1"][c % 64])
        assert np.allclose(g, ref, atol=1e-15, rtol=1e-14)
        assert np.allclose(dg, (1 - np.tanh(z) ** 2) * a["emb00_W0"][c % 32], atol=1e-14)


def test_embedding_derivatives_match_differences(cu_stress_path):
    m = oracle.Model(cu_stress_path)
    h = 1e-5
    for s in [0.02, 0.2, 0.55]:
        g, dg, d2g = m.embed(0, 0, s)
        gp, dgp, _ = m.embed(0, 0, s + h)
        gm, dgm, _ = m.embed(0, 0, s - h)
        assert np.allclose((gp - gm) / (2 * h), dg, atol=1e-8)
        assert np.allclose((dgp - dgm) / (2 * h), d2g, atol=1e-7)
    # and the network is not trivially linear for this model
    assert np.abs(m.embed(0, 0, 0.3)[2]).max() > 1e-2


# ------------------------------------------------------------ fitting net
def test_fitting_reduces_to_closed_form(tmp_path):
    # hidden layers 2 and 3 with W = 0: z_k = z_{k-1} + tanh(b_k), so
    # E = (tanh(D W1 + b1) + tanh(b2) + tanh(b3)) . w + b
    def mut(a):
        a["fit0_W1"][:] = 0
        a["fit0_W2"][:] = 0
    m, a = _special_model(tmp_path, "fit.model", mut)
    D = np.random.default_rng(1).normal(size=2048) * 0.05
    E, _ = m.fit(0, D)
    z = np.tanh(D @ a["fit0_W0"] + a["fit0_b0"]) + np.tanh(a["fit0_b1"]) + np.tanh(a["fit0_b2"])
    ref = z @ a["fit0_wout"] + a["fit0_bout"][0]
    assert abs(E - ref) < 1e-12 * max(1, abs(ref))


def test_fitting_gradient_matches_differences(cu_stress_path):
    m = oracle.Model(cu_stress_path)
    rng = np.random.default_rng(2)
    D = rng.normal(size=2048) * 0.02
    E, dD = m.fit(0, D)
    h = 1e-6
    for k in rng.choice(2048, 12, replace=False):
        e = np.zeros(2048)
        e[k] = h
        fd = (m.fit(0, D + e)[0] - m.fit(0, D - e)[0]) / (2 * h)
        assert abs(fd - dD[k]) < 1e-7 * max(1, abs(dD[k]))


# ------------------------------------------------------------ Sec. 3.2 table
def test_hermite5_exact_on_quintics():
    rng = np.random.default_rng(3)
    for _ in range(20):
        c = rng.normal(size=6)
        h = rng.uniform(0.005, 0.5)
        p = np.polynomial.Polynomial(c)
        y0 = [p(0), p.deriv(1)(0), p.deriv(2)(0)]
        y1 = [p(h), p.deriv(1)(h), p.deriv(2)(h)]
        a = oracle.hermite5(y0, y1, h)
        # compare h^k-scaled coefficients: the data fix a_k only to 1e-16/h^k
        sc = h ** np.arange(6)
        assert np.allclose(a * sc, c * sc, rtol=0, atol=1e-13 * np.abs(c * sc).max())
        # and reproduces it anywhere on the interval
        t = np.linspace(0, h, 7)
        assert np.allclose(np.polynomial.Polynomial(a)(t), p(t), rtol=1e-11, atol=1e-11)


def test_table_matches_net_at_nodes(cu_stress_path):
    m = oracle.Model(cu_stress_path)
    tab = oracle.Table(m, TABLE_H, CU_SMAX)
    assert tab.n == 200
    for k in [0, 1, 17, 40, 66, 150, 199]:
        x = k * TABLE_H
        g, dg, _ = m.embed(0, 0, x)
        for eps in [0.0, 1e-12]:
            tg, tdg, out = tab.eval(0, 0, x + eps)
            assert not out
            assert np.allclose(tg, g, atol=1e-12)
            assert np.allclose(tdg, dg, atol=1e-9)
        # left limit equals right limit (value, slope)
        tg_l, tdg_l, _ = tab.eval(0, 0, x - 1e-12) if k else tab.eval(0, 0, x)
        assert np.allclose(tg_l, g, atol=1e-10) and np.allclose(tdg_l, dg, atol=1e-6)
    assert tab.eval(0, 0, 2.01)[2]  # beyond n*h: reported out of range


def test_table_converges_sixth_order(tmp_path):
    # a model with large weights so the truncation error is far above rounding
    p = tmp_path / "std2.model"
    inputs.write_seeded_model(p, inputs.COPPER_SPEC, seed=0, std=2.0)
    m = oracle.Model(p)
    errs = []
    for h in [0.02, 0.01, 0.005]:
        tab = oracle.Table(m, h, 0.4)
        mid = (np.arange(tab.n) + 0.5) * h  # Hermite error peaks mid-interval
        errs.append(max(np.abs(tab.eval(0, 0, v)[0] - m.embed(0, 0, v)[0]).max() for v in mid))
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    # an O(h^6) method loses a factor 2^6 = 64 per halving (the first halving
    # is still pre-asymptotic); an O(h^4) or O(h^5) error would give 16 or 32
    assert 40 < ratios[0] < 90 and 55 < ratios[1] < 73, (errs, ratios)


def test_extrapolation_region_pins(tmp_path):
    # intervals of width h up to s_max, then of width H = 10 h up to s_ext:
    # the first region is the plain table's, bit for bit; the table equals
    # the net at every node of both regions (both sides of the boundary);
    # the coarse region converges at sixth order in H
    p = tmp_path / "std2.model"
    inputs.write_seeded_model(p, inputs.COPPER_SPEC, seed=0, std=2.0)
    m = oracle.Model(p)
    plain = oracle.Table(m, 0.01, 0.3)
    ext = oracle.Table(m, 0.01, 0.3, s_ext=0.75, ext_stride=10)
    assert (plain.n, ext.n_fine, ext.n, ext.H) == (30, 30, 35, 0.1)
    assert np.array_equal(ext.coeffs()[:30], plain.coeffs())
    nodes = ext.nodes()
    assert np.allclose(nodes[-1], 0.8) and np.allclose(np.diff(nodes), ext.widths())
    for k, x in enumerate(nodes):
        g, dg, _ = m.embed(0, 0, x)
        for side in ([-1e-12] if k else []) + [0.0] + ([1e-12] if k < ext.n else []):
            tg, tdg, out = ext.eval(0, 0, x + side)
            assert not out
            assert np.allclose(tg, g, atol=1e-10) and np.allclose(tdg, dg, atol=1e-6), (k, side)
    assert ext.eval(0, 0, 0.81)[2] and not ext.eval(0, 0, 0.79)[2]
    # coarse region error at interval midpoints: O(H^6) (64 per halving)
    errs = []
    for stride in (8, 4, 2):
        t = oracle.Table(m, 0.0025, 0.3, s_ext=0.62, ext_stride=stride)
        mid = (t.nodes()[t.n_fine:-1] + t.nodes()[t.n_fine + 1:]) / 2
        errs.append(max(np.abs(t.eval(0, 0, v)[0] - m.embed(0, 0, v)[0]).max() for v in mid))
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert 45 < ratios[0] < 80 and 55 < ratios[1] < 73, (errs, ratios)


def test_extrapolation_region_evaluation(stress):
    # a table whose fine region ends below the nearest-neighbor s of copper
    # (s ~ 0.34): those pairs use the coarse intervals.  Forces stay the
    # exact negative gradient of that table's energy, and the energy is
    # close to the untabulated model's within the coarse interpolation error
    m, _ = stress
    tab = oracle.Table(m, TABLE_H, 0.3, s_ext=2.0, ext_stride=10)
    assert tab.n == 30 + 17
    x, t, box = inputs.fcc_copper(3, sigma=0.1, seed=13)
    a = _ev(m, tab, x, t, box)
    b = _ev(m, None, x, t, box)
    assert a["status"] == 0
    d = np.zeros_like(x)
    for i, c in [(0, 0), (5, 1), (33, 2)]:
        for sgn in (1, -1):
            d[i, c] = sgn * 1e-5
            e = _ev(m, tab, x + d, t, box)["energy"]
            d[i, c] = 0.0
            if sgn > 0:
                ep = e
            else:
                fd = -(ep - e) / 2e-5
        assert abs(fd - a["force"][i, c]) < 1e-6 * max(1.0, abs(fd)), (i, c, fd)
    assert abs(a["energy"] - b["energy"]) / len(x) < 1e-3 * np.abs(b["atom_energy"]).mean()


# ------------------------------------------------------------ neighbors
def test_fcc_shell_counts_golden():
    rows = np.loadtxt(os.path.join(HERE, "golden", "fcc_shells.txt"), dtype=int)
    counts = dict(rows)
    # brute force over FCC lattice vectors (integer coordinates in units of
    # a/2 with even coordinate sum)
    r = np.arange(-6, 7)
    X, Y, Z = np.meshgrid(r, r, r, indexing="ij")
    ok = ((X + Y + Z) % 2 == 0)
    n2 = (X * X + Y * Y + Z * Z)[ok]  # |v|^2 in (a/2)^2 units = 2k
    for k, c in counts.items():
        assert (n2 == 2 * k).sum() == c
    # perfect Cu lattice: every atom has exactly 176 neighbors within 8 A
    x, _, box = inputs.fcc_copper(6, a=3.634, sigma=0.0)
    nb = oracle.neighbors(x, box, 8.0, method=1)
    per = np.bincount(nb[:, 0], minlength=len(x))
    assert (per == sum(c for k, c in counts.items() if 3.634 * np.sqrt(k / 2) < 8.0)).all()
    assert (per == 176).all()


@pytest.mark.parametrize("ncell,rlist", [((3, 3, 3), 4.0), ((2, 3, 4), 5.0),
                                         ((3, 3, 3), 10.0), ((5, 5, 5), 10.0)])
def test_cell_list_equals_brute_force(ncell, rlist):
    x, _, box = inputs.fcc_copper(ncell, sigma=0.3, seed=11)
    x = x + np.random.default_rng(1).uniform(-30, 30, size=3)  # unwrapped input
    if min(np.diag(box)) < rlist:
        with pytest.raises(oracle.OracleError):
            oracle.neighbors(x, box, rlist, method=1)
        return
    a = oracle.neighbors(x, box, rlist, method=0)
    b = oracle.neighbors(x, box, rlist, method=1)
    assert len(a) > 0 and np.array_equal(a, b)
    # symmetric: (i, j, n) present iff (j, i, -n) present
    rev = np.concatenate([a[:, 1:2], a[:, 0:1], -a[:, 2:]], axis=1)
    rev = rev[np.lexsort(rev.T[::-1])]
    assert np.array_equal(rev, a)


# ------------------------------------------------------------ energy / forces
def _cluster(n=24, seed=4, spacing=2.6):
    # a free cluster: atoms on a jittered cubic grid inside a huge box
    rng = np.random.default_rng(seed)
    g = np.stack(np.meshgrid(*[np.arange(3)] * 3, indexing="ij"), -1).reshape(-1, 3)[:n]
    x = g * spacing + rng.normal(0, 0.15, size=(n, 3)) + 40.0
    box = np.diag([100.0, 100.0, 100.0])
    return x, np.zeros(n, np.int32), box


@pytest.fixture(scope="module")
def stress(cu_stress_path):
    m = oracle.Model(cu_stress_path)
    return m, oracle.Table(m, TABLE_H, CU_SMAX)


def _ev(m, tab, x, t, box, **kw):
    return oracle.evaluate(m, tab, CU_RC, CU_RCS, CU_SEL, x, t, box, **kw)


def _dE(rp, rm):
    # energy difference summed atom by atom: the per-atom energies are large
    # and nearly constant, so differencing the totals would lose ~1e-12 eV
    return float(np.sum(rp["atom_energy"] - rm["atom_energy"]))


@pytest.mark.parametrize("tabulated", [False, True])
def test_forces_are_minus_gradient(stress, tabulated):
    m, tab = stress
    tab = tab if tabulated else None
    x, t, box = inputs.fcc_copper(3, sigma=0.1, seed=5)
    r = _ev(m, tab, x, t, box)
    assert np.sqrt((r["force"] ** 2).mean()) > 1e-2  # non-trivial forces
    # step 5e-5 A balances truncation (~h^2) against the ~1e-12 eV rounding
    # noise of the per-atom energies of this large-weight model (~1/h)
    h = 5e-5
    rng = np.random.default_rng(6)
    for i in rng.choice(len(x), 5, replace=False):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = -_dE(_ev(m, tab, xp, t, box), _ev(m, tab, xm, t, box)) / (2 * h)
            assert abs(fd - r["force"][i, a]) < 1e-7, (i, a, fd, r["force"][i, a])


def test_total_force_zero_and_virial_symmetric(stress):
    m, tab = stress
    x, t, box = inputs.fcc_copper(4, sigma=0.1, seed=7)
    r = _ev(m, tab, x, t, box)
    assert np.abs(r["force"].sum(0)).max() < 1e-11
    V = r["virial"]
    assert np.abs(V - V.T).max() < 1e-10 * np.abs(V).max()


def test_virial_is_strain_derivative(stress):
    m, tab = stress
    # periodic box: diagonal strain of box and positions
    x, t, box = inputs.fcc_copper(3, sigma=0.1, seed=8)
    V = _ev(m, tab, x, t, box)["virial"]
    h = 1e-6
    for a in range(3):
        S = np.eye(3)
        S[a, a] += h
        rp = _ev(m, tab, x @ S.T, t, box @ S.T)
        S[a, a] -= 2 * h
        rm = _ev(m, tab, x @ S.T, t, box @ S.T)
        assert abs(-_dE(rp, rm) / (2 * h) - V[a, a]) < 1e-7 * max(1, abs(V[a, a]))
    # free cluster: any strain of the positions, off-diagonal included
    xc, tc, bc = _cluster()
    Vc = _ev(m, tab, xc, tc, bc)["virial"]
    c0 = xc.mean(0)
    for a in range(3):
        for b in range(3):
            S = np.zeros((3, 3))
            S[a, b] = h
            rp = _ev(m, tab, c0 + (xc - c0) @ (np.eye(3) + S).T, tc, bc)
            rm = _ev(m, tab, c0 + (xc - c0) @ (np.eye(3) - S).T, tc, bc)
            # dE/d eps_ab = sum g_a r_b = -V[b, a]
            assert abs(-_dE(rp, rm) / (2 * h) - Vc[b, a]) < 1e-7 * max(1, np.abs(Vc).max())


def test_energy_invariances(stress):
    m, tab = stress
    x, t, box = inputs.fcc_copper(3, sigma=0.15, seed=9)
    L = box[0, 0]
    r0 = _ev(m, tab, x, t, box)
    E0, F0 = r0["energy"], r0["force"]
    tol = 1e-12 * abs(E0)
    # translation
    r = _ev(m, tab, x + np.array([1.7, -0.3, 12.9]), t, box)
    assert abs(r["energy"] - E0) < tol and np.allclose(r["force"], F0, atol=1e-10)
    # cubic symmetries of the periodic box: axis permutation and reflection
    r = _ev(m, tab, x[:, [1, 2, 0]], t, box)
    assert abs(r["energy"] - E0) < tol and np.allclose(r["force"], F0[:, [1, 2, 0]], atol=1e-10)
    xr = x.copy()
    xr[:, 0] = L - xr[:, 0]
    r = _ev(m, tab, xr, t, box)
    Fr = F0.copy()
    Fr[:, 0] *= -1
    assert abs(r["energy"] - E0) < tol and np.allclose(r["force"], Fr, atol=1e-10)
    # same-type permutation: energy invariant, forces permuted
    perm = np.random.default_rng(3).permutation(len(x))
    r = _ev(m, tab, x[perm], t, box)
    assert abs(r["energy"] - E0) < tol and np.allclose(r["force"], F0[perm], atol=1e-10)
    assert np.allclose(r["atom_energy"], r0["atom_energy"][perm], atol=1e-12)
    # arbitrary rotation of a free cluster
    xc, tc, bc = _cluster()
    rc0 = _ev(m, tab, xc, tc, bc)
    Q = inputs._random_rotation(np.random.default_rng(10))
    c0 = xc.mean(0)
    rc1 = _ev(m, tab, c0 + (xc - c0) @ Q.T, tc, bc)
    assert abs(rc1["energy"] - rc0["energy"]) < 1e-12 * abs(rc0["energy"])
    assert np.allclose(rc1["force"], rc0["force"] @ Q.T, atol=1e-10)


def test_isolated_atom_is_fitting_at_zero(stress):
    m, tab = stress
    x = np.array([[1.0, 1.0, 1.0], [20.0, 20.0, 20.0]])
    box = np.diag([40.0, 40.0, 40.0])
    r = _ev(m, tab, x, np.zeros(2, np.int32), box)
    E0, _ = m.fit(0, np.zeros(2048))
    assert np.allclose(r["atom_energy"], E0, atol=1e-14)
    assert np.abs(r["force"]).max() == 0.0


def test_two_types_water(water_model_path):
    m = oracle.Model(water_model_path)
    assert m.ntypes == 2 and m.M == 100
    tab = oracle.Table(m, TABLE_H, 1.25)
    x, t, box = inputs.water_like(16, L=7.82, seed=3)  # 48 atoms, same density
    r = oracle.evaluate(m, tab, 6.0, 0.5, [46, 92], x, t, box)
    ru = oracle.evaluate(m, None, 6.0, 0.5, [46, 92], x, t, box)
    assert abs(r["energy"] - ru["energy"]) / len(x) < 1e-7
    # type swap is not a symmetry: relabelling changes the energy
    r2 = oracle.evaluate(m, tab, 6.0, 0.5, [46, 92], x, 1 - t, box, check=False)
    assert abs(r2["energy"] - r["energy"]) > 1e-3
    # FD force on an O and an H
    h = 1e-5
    for i in [0, 20]:
        xp, xm = x.copy(), x.copy()
        xp[i, 2] += h
        xm[i, 2] -= h
        fd = -_dE(oracle.evaluate(m, tab, 6.0, 0.5, [46, 92], xp, t, box),
                  oracle.evaluate(m, tab, 6.0, 0.5, [46, 92], xm, t, box)) / (2 * h)
        assert abs(fd - r["force"][i, 2]) < 1e-7


@pytest.mark.parametrize("tabulated", [False, True])
def test_two_types_water_virial_and_total_force(water_model_path, tabulated):
    # the two-type path (per type-pair nets or tables, sel sections [46, 92],
    # two fitting nets): zero total force, a symmetric virial, and the virial
    # as the energy's derivative under a diagonal strain of box and positions
    m = oracle.Model(water_model_path)
    tab = oracle.Table(m, TABLE_H, 1.25) if tabulated else None
    x, t, box = inputs.water_like(16, L=7.82, seed=3)  # 48 atoms
    ev = lambda xx, bb: oracle.evaluate(m, tab, 6.0, 0.5, [46, 92], xx, t, bb)
    r = ev(x, box)
    F, V = r["force"], r["virial"]
    assert np.abs(F.sum(0)).max() < 1e-10 * max(1.0, np.abs(F).max())
    assert np.abs(V - V.T).max() < 1e-10 * max(1.0, np.abs(V).max())
    h = 1e-6
    for a in range(3):
        S = np.eye(3)
        S[a, a] += h
        rp = ev(x @ S.T, box @ S.T)
        S[a, a] -= 2 * h
        rm = ev(x @ S.T, box @ S.T)
        assert abs(-_dE(rp, rm) / (2 * h) - V[a, a]) < 1e-7 * max(1, abs(V[a, a]))


def test_sel_overflow_and_table_range_reported(stress):
    m, tab = stress
    x, t, box = inputs.fcc_copper(3, sigma=0.0)
    r = oracle.evaluate(m, tab, CU_RC, CU_RCS, 100, x, t, box, check=False)
    assert r["status"] == 5 and r["n_sel"] == len(x)
    x2 = x.copy()
    x2[1] = x2[0] + np.array([0.45, 0, 0])  # r = 0.45 A -> s = 1/0.45 > 2
    r = oracle.evaluate(m, tab, CU_RC, CU_RCS, CU_SEL, x2, t, box, check=False)
    assert r["status"] == 6 and r["n_range"] >= 2


def test_sel_overflow_per_neighbor_type_water(water_model_path):
    # N_m is sectioned by neighbor type (sel [46, 92]): an atom overflows when
    # its count of one type passes that type's section.  The counts come from
    # a minimum-image brute force here (rc = 6 < L / 2), independent of the
    # oracle's cell list; the oracle must flag exactly the atoms they flag.
    m = oracle.Model(water_model_path)
    tab = oracle.Table(m, TABLE_H, 1.25)
    x, t, box = inputs.water_like(64, L=12.417, seed=3)
    L = np.diag(box)
    d = x[None, :, :] - x[:, None, :]
    d -= L * np.round(d / L)
    r2 = (d ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    within = r2 < 6.0 ** 2
    cnt = np.stack([(within & (t[None, :] == k)).sum(1) for k in (0, 1)], 1)
    r = oracle.evaluate(m, tab, 6.0, 0.5, [46, 92], x, t, box)
    assert r["status"] == 0 and cnt[:, 0].max() <= 46 and cnt[:, 1].max() <= 92
    for k in (0, 1):
        sel = [46, 92]
        sel[k] = int(cnt[:, k].max()) - 1
        r = oracle.evaluate(m, tab, 6.0, 0.5, sel, x, t, box, check=False)
        assert r["status"] == 5 and r["n_sel"] == int((cnt[:, k] > sel[k]).sum()), (k, r["n_sel"])


def test_subset_matches_full(stress):
    m, tab = stress
    x, t, box = inputs.fcc_copper(4, sigma=0.1, seed=12)
    r = _ev(m, tab, x, t, box)
    ie = np.array([0, 5, 77, 255])
    jf = np.array([3, 100, 200])
    e, f = oracle.eval_subset(m, tab, CU_RC, CU_RCS, CU_SEL, x, t, box, ie, jf)
    assert np.allclose(e, r["atom_energy"][ie], atol=1e-13)
    assert np.allclose(f, r["force"][jf], atol=1e-12)


def test_tabulation_error_small(stress):
    m, tab = stress
    x, t, box = inputs.fcc_copper(3, sigma=0.1, seed=13)
    a = _ev(m, tab, x, t, box)
    b = _ev(m, None, x, t, box)
    assert abs(a["energy"] - b["energy"]) / len(x) < 1e-7
    assert rmse(a["force"], b["force"]) < 1e-6


# ------------------------------------------------------------ MD (Sec. 4)
def test_md_energy_conservation_and_reversibility(stress):
    m, tab = stress
    x, t, box = inputs.fcc_copper(3, sigma=0.05, seed=14)
    masses = np.array([inputs.MASS_CU])
    v = inputs.maxwell_velocities(np.full(len(x), inputs.MASS_CU), 330.0, seed=2)
    drift = []
    for dt in [1.0, 0.5]:
        n = int(round(20 / dt))
        _, _, _, th = oracle.md(m, tab, CU_RC, CU_RCS, CU_SEL, x, v, t, masses, box, dt, n)
        etot = th[:, 0] + th[:, 1]
        drift.append(np.abs(etot - etot[0]).max())
        assert abs(th[0, 2] - 330.0) < 1e-9
    # Verlet error falls as dt^2
    assert drift[1] < drift[0] / 2.5, drift
    # time reversal: run, flip v, run back
    x1, v1, _, _ = oracle.md(m, tab, CU_RC, CU_RCS, CU_SEL, x, v, t, masses, box, 1.0, 10)
    x2, v2, _, _ = oracle.md(m, tab, CU_RC, CU_RCS, CU_SEL, x1, -v1, t, masses, box, 1.0, 10)
    assert np.abs(x2 - x).max() < 1e-9 and np.abs(v2 + v).max() < 1e-10


def test_md_two_masses_water(water_model_path):
    # velocity-Verlet with a mass per type (O 15.999, H 1.008 amu).  One step
    # from rest moves every atom by dt^2/2 * F/m (the unit factor from CODATA:
    # 1 eV/A/amu in A/fs^2), which pins each type's mass in the kicks; then
    # the energy drift falls as dt^2 and a run reversed returns to its start
    m = oracle.Model(water_model_path)
    tab = oracle.Table(m, TABLE_H, 2.0)
    x, t, box = inputs.water_like(16, L=7.82, seed=3)  # 48 atoms
    masses = np.array([inputs.MASS_O, inputs.MASS_H])
    mass = masses[t]
    kappa = 1.602176634e-19 / 1e-10 / 1.66053906660e-27 * 1e-20  # (eV/A/amu) -> A/fs^2
    f0 = oracle.evaluate(m, tab, 6.0, 0.5, [46, 92], x, t, box)["force"]
    dt = 0.05
    x1, _, _, _ = oracle.md(m, tab, 6.0, 0.5, [46, 92], x, np.zeros_like(x), t, masses, box, dt, 1)
    L = np.diag(box)
    dx = (x1 - x) - L * np.round((x1 - x) / L)
    want = 0.5 * dt * dt * kappa * f0 / mass[:, None]
    assert np.abs(dx - want).max() < 1e-9 * np.abs(want).max(), np.abs(dx - want).max()
    v = inputs.maxwell_velocities(mass, 30.0, seed=5)
    drift = []
    for dt in [0.1, 0.05, 0.025]:
        _, _, _, th = oracle.md(m, tab, 6.0, 0.5, [46, 92], x, v, t, masses, box, dt,
                                int(round(1.0 / dt)))
        etot = th[:, 0] + th[:, 1]
        drift.append(np.abs(etot - etot[0]).max())
    assert 3.5 < drift[0] / drift[1] < 4.5 and 3.5 < drift[1] / drift[2] < 4.5, drift
    x1, v1, _, _ = oracle.md(m, tab, 6.0, 0.5, [46, 92], x, v, t, masses, box, 0.1, 10)
    x2, v2, _, _ = oracle.md(m, tab, 6.0, 0.5, [46, 92], x1, -v1, t, masses, box, 0.1, 10)
    assert np.abs(x2 - x).max() < 1e-9 and np.abs(v2 + v).max() < 1e-10


# ------------------------------------------------------------------ Sec. 3.5 tanh table
def test_tanh_table_pins():
    import math
    oracle.set_tanh_table(True)
    try:
        h = 1.0 / 128
        for k in [0, 1, 77, 500, 1023]:
            x = k * h
            t, d = oracle.act(x)
            assert abs(t - math.tanh(x)) < 1e-15           # exact at the nodes
            assert abs(d - (1 - math.tanh(x) ** 2)) < 1e-15  # slope matched at the left node
            t1, _ = oracle.act(x + h * (1 - 1e-12))
            assert abs(t1 - math.tanh(x + h)) < 1e-12       # value matched at the right node
        xs = np.linspace(0.0, 7.999, 40001)
        err = max(abs(oracle.act(x)[0] - math.tanh(x)) for x in xs)
        assert err < 3e-8, err  # third-order error of a quadratic at h = 1/128
        for x in [0.3, 2.7, 7.5]:
            assert oracle.act(-x)[0] == -oracle.act(x)[0]  # odd
            assert oracle.act(-x)[1] == oracle.act(x)[1]
            # the stored derivative is the derivative of the table polynomial
            e = 1e-6
            fd = (oracle.act(x + e)[0] - oracle.act(x - e)[0]) / (2 * e)
            assert abs(fd - oracle.act(x)[1]) < 1e-8
        assert oracle.act(8.0) == (1.0, 0.0) and oracle.act(-9.5) == (-1.0, 0.0)
    finally:
        oracle.set_tanh_table(False)
    assert oracle.act(0.3)[0] == math.tanh(0.3)


def test_fit_gradient_with_tanh_table(cu_stress_path):
    # forces stay the exact gradient of the energy the table gives
    m = oracle.Model(cu_stress_path)
    rng = np.random.default_rng(3)
    D = rng.normal(scale=0.05, size=m.din)
    oracle.set_tanh_table(True)
    try:
        E, dD = m.fit(0, D)
        for j in rng.choice(m.din, 6, replace=False):
            e = 1e-6
            Dp, Dm = D.copy(), D.copy()
            Dp[j] += e
            Dm[j] -= e
            fd = (m.fit(0, Dp)[0] - m.fit(0, Dm)[0]) / (2 * e)
            assert abs(fd - dD[j]) < 2e-6 * max(1.0, abs(dD[j])), (j, fd, dD[j])
        E0, _ = m.fit(0, D)
    finally:
        oracle.set_tanh_table(False)
    Ex, _ = m.fit(0, D)
    assert E0 == E and abs(E - Ex) < 1e-4 * max(1.0, abs(Ex))
