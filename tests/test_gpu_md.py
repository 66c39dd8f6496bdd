"""Velocity-Verlet MD on the GPU (Sec. 4) against the oracle's MD, plus energy
conservation, checkpoint/resume identity and the list-skin guard."""
import numpy as np
import pytest

import oracle
from paper_2201_01446_gb300 import inputs
from conftest import CU_RC, CU_RCS, CU_SEL, CU_SMAX, PARITY_LOG, TABLE_H, rmse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    from paper_2201_01446_gb300 import dp as _dp
    return _dp


@pytest.fixture(scope="module")
def stress(dp, cu_stress_path):
    o = dp.dp_options_default()
    h = dp.dp_create(cu_stress_path, 1, CU_RC, CU_RCS, [CU_SEL], options=o, stream=None)
    m = oracle.Model(cu_stress_path)
    yield h, m, oracle.Table(m, TABLE_H, CU_SMAX)
    dp.dp_destroy(h)


def _system(n=4, seed=14):
    x, t, box = inputs.fcc_copper(n, sigma=0.05, seed=seed)
    v = inputs.maxwell_velocities(np.full(len(x), inputs.MASS_CU), 330.0, seed=2)
    return x, v, t, box


def test_md_matches_oracle_trajectory(dp, stress):
    h, m, tab = stress
    x, v, t, box = _system()
    s = dp.dp_system_create(h, x, v, t, [inputs.MASS_CU], box)
    try:
        th = dp.dp_md_step(h, s, 12, 1.0, thermo=True)  # crosses a list rebuild at step 10
        xg, vg, fg = dp.dp_system_get(h, s, len(x))
    finally:
        dp.dp_system_destroy(s)
    xo, vo, fo, tho = oracle.md(m, tab, CU_RC, CU_RCS, CU_SEL, x, v, t, [inputs.MASS_CU], box,
                                1.0, 12)
    L = np.diag(box)
    dx = (xg - xo) - L * np.round((xg - xo) / L)
    assert np.abs(dx).max() < 1e-6
    assert np.abs(vg - vo).max() < 1e-7
    assert rmse(fg, fo) < 1e-5
    # thermo: kinetic and potential energy per step.  This large-weight model
    # has |E_i| ~ 27 eV, so FP32 rounding (~5e-7 relative, correlated across a
    # near-perfect lattice) sets a relative bound on the potential energy
    assert np.abs(th[:, 1] - tho[1:, 0]).max() < 1e-6 * len(x)
    assert np.abs(th[:, 2] - tho[1:, 1]).max() < 2e-6 * np.abs(tho[1:, 1]).max()
    assert np.array_equal(th[:, 0], np.arange(1, 13))


@pytest.mark.parametrize("fit,embed", [(0, 0), (4, 2)])
def test_md_two_masses_water_matches_oracle(dp, water_model_path, fit, embed):
    # two-type water (O 15.999, H 1.008 amu) on the stress model, whose H atoms
    # feel ~10 eV/A: 12 steps of 0.1 fs (crossing the list rebuild at step 10)
    # against the oracle's MD.  A mass taken from the wrong type would move an
    # H atom ~0.1 A off; FP32 forces move it ~1e-6 A
    m = oracle.Model(water_model_path)
    tab = oracle.Table(m, TABLE_H, 2.0)
    x, t, box = inputs.water_like(64, L=12.417, seed=3)
    masses = [inputs.MASS_O, inputs.MASS_H]
    v = inputs.maxwell_velocities(np.where(t == 0, inputs.MASS_O, inputs.MASS_H), 30.0, seed=5)
    o = dp.dp_options_default()
    o.fit_precision = fit
    o.embed_precision = embed
    o.s_max = 2.0
    h = dp.dp_create(water_model_path, 2, 6.0, 0.5, [46, 92], options=o, stream=None)
    try:
        s = dp.dp_system_create(h, x, v, t, masses, box)
        dp.dp_md_step(h, s, 12, 0.1)
        xg, vg, fg = dp.dp_system_get(h, s, len(x))
        dp.dp_system_destroy(s)
    finally:
        dp.dp_destroy(h)
    xo, vo, fo, _ = oracle.md(m, tab, 6.0, 0.5, [46, 92], x, v, t, masses, box, 0.1, 12)
    L = np.diag(box)
    dx = (xg - xo) - L * np.round((xg - xo) / L)
    moved = (xo - x) - L * np.round((xo - x) / L)
    PARITY_LOG.append(dict(case=f"water MD 12 x 0.1 fs fit {fit} embed {embed}", natoms=len(x),
                           max_dx=float(np.abs(dx).max()), max_dv=float(np.abs(vg - vo).max()),
                           force_rmse=rmse(fg, fo), max_moved=float(np.abs(moved).max())))
    assert np.abs(moved).max() > 1e-2  # the check below resolves the motion
    assert np.abs(dx).max() < 1e-5
    assert np.abs(vg - vo).max() < 1e-5
    assert rmse(fg, fo) < 3e-5 * float(np.sqrt((fo ** 2).mean()))


def test_checkpoint_resume_bitwise(dp, stress, tmp_path):
    h, _, _ = stress
    x, v, t, box = _system(5, seed=15)
    a = dp.dp_system_create(h, x, v, t, [inputs.MASS_CU], box)
    dp.dp_md_step(h, a, 20, 1.0)
    xa, va, fa = dp.dp_system_get(h, a, len(x))
    dp.dp_system_destroy(a)
    b = dp.dp_system_create(h, x, v, t, [inputs.MASS_CU], box)
    dp.dp_md_step(h, b, 10, 1.0)
    dp.dp_state_save(h, b, tmp_path / "st.bin")
    dp.dp_system_destroy(b)
    c = dp.dp_state_load(h, tmp_path / "st.bin")
    assert dp.dp_system_step(c) == 10
    dp.dp_md_step(h, c, 10, 1.0)
    xc, vc, fc = dp.dp_system_get(h, c, len(x))
    dp.dp_system_destroy(c)
    assert np.array_equal(xa, xc) and np.array_equal(va, vc) and np.array_equal(fa, fc)


def test_energy_conservation(dp, stress):
    # Verlet energy error ~dt^2.  FP32 rounding puts ~5e-4 eV of noise on this
    # model's total energy (|E| ~ 7e3 eV), so the steps are large enough
    # (8 and 4 fs over 80 fs) for the integrator error to stand well above it
    h, m, tab = stress
    x, v, t, box = _system(4, seed=16)
    drift = []
    for dt in (8.0, 4.0):
        s = dp.dp_system_create(h, x, v, t, [inputs.MASS_CU], box)
        th = dp.dp_md_step(h, s, int(round(80 / dt)), dt, thermo=True)
        dp.dp_system_destroy(s)
        e = th[:, 1] + th[:, 2]
        drift.append(np.abs(e - e[0]).max())
    assert drift[1] < drift[0] / 2.5, drift
    _, _, _, tho = oracle.md(m, tab, CU_RC, CU_RCS, CU_SEL, x, v, t, [inputs.MASS_CU], box, 8.0, 10)
    eo = tho[1:, 0] + tho[1:, 1]
    ref = np.abs(eo - eo[0]).max()
    assert abs(drift[0] - ref) < 0.2 * ref + 1e-3, (drift[0], ref)


def test_skin_violation_reported(dp, stress):
    h, _, _ = stress
    x, v, t, box = _system(4, seed=17)
    s = dp.dp_system_create(h, x, v * 60.0, t, [inputs.MASS_CU], box)  # ~1 A/fs
    try:
        with pytest.raises(dp.DPError) as e:
            dp.dp_md_step(h, s, 5, 1.0)
        assert e.value.code == 10
    finally:
        dp.dp_system_destroy(s)


@pytest.mark.parametrize("prec", [0, 2])
def test_md_graph_replay_bitwise(dp, cu_stress_path, prec):
    # plain MD steps replayed as one captured CUDA graph give bitwise the
    # launches' results, across list rebuilds, and count the same launches
    import time
    x, v, t, box = _system(4, seed=16)
    out = {}
    for graphs in (0, 1):
        o = dp.dp_options_default()
        o.md_graphs = graphs
        o.fit_precision = prec
        o.embed_precision = prec
        h = dp.dp_create(cu_stress_path, 1, CU_RC, CU_RCS, [CU_SEL], options=o, stream=None)
        try:
            s = dp.dp_system_create(h, x, v, t, [inputs.MASS_CU], box)
            dp.dp_md_step(h, s, 3, 1.0)
            l0 = dp.dp_stats(h, s)["kernel_launches"]
            t0 = time.perf_counter()
            dp.dp_md_step(h, s, 22, 1.0)  # rebuilds at steps 10 and 20
            xg, vg, fg = dp.dp_system_get(h, s, len(x))
            dt = time.perf_counter() - t0
            out[graphs] = (xg, vg, fg, dp.dp_stats(h, s)["kernel_launches"] - l0, dt)
            dp.dp_system_destroy(s)
        finally:
            dp.dp_destroy(h)
    a, b = out[0], out[1]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert a[3] == b[3], (a[3], b[3])
    PARITY_LOG.append(dict(case=f"md graphs 256 atoms prec {prec}", ms_per_step_launches=a[4] / 22e-3,
                           ms_per_step_graphs=b[4] / 22e-3))


def test_md_graph_replay_after_set_params(dp, cu_stress_path):
    # new parameters between MD calls: replayed graphs must see them (the
    # output bias is a launch parameter), so graphs and launches still agree
    x, v, t, box = _system(4, seed=17)
    out = {}
    for graphs in (0, 1):
        o = dp.dp_options_default()
        o.md_graphs = graphs
        o.fit_precision = 2
        o.embed_precision = 2
        h = dp.dp_create(cu_stress_path, 1, CU_RC, CU_RCS, [CU_SEL], options=o, stream=None)
        try:
            s = dp.dp_system_create(h, x, v, t, [inputs.MASS_CU], box)
            dp.dp_md_step(h, s, 5, 1.0)
            fit, tab = dp.dp_get_params(h)
            fit[-1] += 0.25  # output bias: shifts every E_i, not the forces
            fit[:-1] *= 1.01
            dp.dp_set_params(h, fit, None)
            th = dp.dp_md_step(h, s, 3, 1.0, thermo=True)
            dp.dp_md_step(h, s, 4, 1.0)
            xg, vg, fg = dp.dp_system_get(h, s, len(x))
            E, F, V, _ = dp.dp_compute(h, xg, t, box)
            out[graphs] = (xg, vg, fg, th, E)
            dp.dp_system_destroy(s)
        finally:
            dp.dp_destroy(h)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
