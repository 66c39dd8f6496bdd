"""Several systems in one evaluation (dp_compute_batch, the packed launch of
the serving loop): per system the energy, forces and virial are bitwise
those of dp_compute on the system alone; one system against the oracle;
empty and one-atom systems; copper and two-type water; the mode
requirement."""
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


def _tc(dp, path, ntypes=1, rc=CU_RC, rcs=CU_RCS, sel=(CU_SEL,), s_max=CU_SMAX, fit=2):
    o = dp.dp_options_default()
    o.embed_precision = 2
    o.fit_precision = fit
    o.s_max = s_max
    return dp.dp_create(path, ntypes, rc, rcs, list(sel), options=o, stream=None)


def _check_alone(dp, h, systems, tag):
    E, F, V = dp.dp_compute_batch(h, systems)
    for q, (x, t, box) in enumerate(systems):
        Ea, Fa, Va, _ = dp.dp_compute(h, x, t, box)
        # bitwise: the same per-atom and per-tile values, summed in the same order
        assert np.array_equal(F[q], Fa), (tag, q)
        assert E[q] == Ea, (tag, q, E[q], Ea)
        assert np.array_equal(V[q], Va), (tag, q)
    PARITY_LOG.append(dict(case=f"batch vs alone (bitwise): {tag}", systems=len(systems)))
    return E, F, V


@pytest.mark.parametrize("fit", [2, 4])
def test_batch_copper_matches_alone_and_oracle(dp, cu_stress_path, fit):
    h = _tc(dp, cu_stress_path, fit=fit)
    try:
        systems = [inputs.fcc_copper(5, sigma=0.05, seed=1),
                   inputs.fcc_copper((3, 4, 5), sigma=0.15, seed=2),
                   (np.zeros((0, 3)), np.zeros(0, np.int32), np.diag([30.0, 30.0, 30.0])),
                   (np.array([[1.0, 2.0, 3.0]]), np.zeros(1, np.int32), np.diag([40.0] * 3)),
                   inputs.fcc_copper(4, sigma=0.1, seed=3)]
        E, F, V = _check_alone(dp, h, systems, f"Cu 500 + 240 + 0 + 1 + 256, fit {fit}")
        assert E[2] == 0.0 and F[2].shape == (0, 3) and not V[2].any()
        # the 240-atom system (ragged tiles, non-cubic box) against the oracle
        m = oracle.Model(cu_stress_path)
        x, t, box = systems[1]
        r = oracle.evaluate(m, oracle.Table(m, TABLE_H, CU_SMAX), CU_RC, CU_RCS, CU_SEL, x, t, box)
        frms = float(np.sqrt((r["force"] ** 2).mean()))
        assert abs(E[1] - r["energy"]) / len(x) < max(1e-6, 5e-6 * np.abs(r["atom_energy"]).mean())
        assert rmse(F[1], r["force"]) < max(1e-5, 3e-5 * frms)
        assert np.abs(V[1] - r["virial"]).max() < 1e-4 * np.abs(r["virial"]).max() + 1e-9
    finally:
        dp.dp_destroy(h)


def test_batch_water_two_types(dp, water_model_path):
    h = _tc(dp, water_model_path, 2, 6.0, 0.5, (46, 92), 1.25)
    try:
        systems = [inputs.water_like(64, L=12.417, seed=s) for s in (3, 4, 5)]
        _check_alone(dp, h, systems, "3 x water 192")
    finally:
        dp.dp_destroy(h)


def test_batch_needs_tensor_core_embedding(dp, cu_model_path):
    h = dp.dp_create(cu_model_path, 1, CU_RC, CU_RCS, [CU_SEL], options=None, stream=None)
    try:
        with pytest.raises(dp.DPError) as e:
            dp.dp_compute_batch(h, [inputs.fcc_copper(3, sigma=0.05, seed=1)])
        assert e.value.code == 9
    finally:
        dp.dp_destroy(h)


def test_batch_md_matches_alone(dp, cu_stress_path):
    # several systems advanced as one (list rebuilds at steps 10 and 20, plain
    # steps replayed as a graph, then steps with thermo records): each
    # trajectory and each system's records bitwise those it has alone
    h = _tc(dp, cu_stress_path)
    try:
        sys3 = []
        for k, (cells, sig) in enumerate([(4, 0.05), ((3, 4, 5), 0.1), (5, 0.05)]):
            x, t, box = inputs.fcc_copper(cells, sigma=sig, seed=20 + k)
            v = inputs.maxwell_velocities(np.full(len(x), inputs.MASS_CU), 330.0, seed=30 + k)
            sys3.append((x, v, t, box))
        sb = dp.dp_system_create_batch(h, sys3, [inputs.MASS_CU])
        try:
            assert dp.lib.dp_system_batch_size(sb) == 3
            dp.dp_md_step(h, sb, 20, 1.0)
            thb = dp.dp_md_step(h, sb, 3, 1.0, thermo=True)
            n = sum(len(s[0]) for s in sys3)
            xb, vb, fb = dp.dp_system_get(h, sb, n)
        finally:
            dp.dp_system_destroy(sb)
        assert thb.shape == (3, 3, 5)
        o = 0
        for q, (x, v, t, box) in enumerate(sys3):
            s = dp.dp_system_create(h, x, v, t, [inputs.MASS_CU], box)
            try:
                assert dp.lib.dp_system_batch_size(s) == 0
                dp.dp_md_step(h, s, 20, 1.0)
                tha = dp.dp_md_step(h, s, 3, 1.0, thermo=True)
                xa, va, fa = dp.dp_system_get(h, s, len(x))
            finally:
                dp.dp_system_destroy(s)
            m = len(x)
            assert np.array_equal(xb[o:o + m], xa) and np.array_equal(vb[o:o + m], va)
            assert np.array_equal(fb[o:o + m], fa)
            assert np.array_equal(thb[:, q], tha), (q, thb[:, q], tha)
            o += m
    finally:
        dp.dp_destroy(h)


def test_batch_errors_and_type_map(dp, cu_stress_path, water_model_path):
    # an over-full system fails the whole call with the sel error; caller
    # types reach the model through the handle's type map, as in dp_compute
    h = _tc(dp, cu_stress_path, sel=(100,))
    try:
        with pytest.raises(dp.DPError) as e:
            dp.dp_compute_batch(h, [inputs.fcc_copper(3, sigma=0.05, seed=1),
                                    inputs.fcc_copper(4, sigma=0.0)])
        assert e.value.code == 5
    finally:
        dp.dp_destroy(h)
    o = dp.dp_options_default()
    o.embed_precision = 2
    o.fit_precision = 2
    o.s_max = 1.25
    # caller types 0 = H, 1 = O mapped onto model types 1, 0
    hm = dp.dp_create(water_model_path, 2, 6.0, 0.5, [46, 92], type_map=[1, 0], options=o,
                      stream=None)
    try:
        sys2 = [inputs.water_like(64, L=12.417, seed=s) for s in (3, 6)]
        swapped = [(x, 1 - t, box) for x, t, box in sys2]
        _check_alone(dp, hm, swapped, "2 x water 192, mapped types")
    finally:
        dp.dp_destroy(hm)


def test_batch_state_file_resume_bitwise(dp, cu_stress_path, tmp_path):
    # a batch system saved between list rebuilds (step 13) and loaded again
    # continues bitwise as the uninterrupted run; the file keeps every system
    h = _tc(dp, cu_stress_path)
    try:
        sys2 = []
        for k, (cells, sig) in enumerate([((3, 4, 5), 0.1), (4, 0.05)]):
            x, t, box = inputs.fcc_copper(cells, sigma=sig, seed=40 + k)
            v = inputs.maxwell_velocities(np.full(len(x), inputs.MASS_CU), 330.0, seed=50 + k)
            sys2.append((x, v, t, box))
        n = sum(len(s[0]) for s in sys2)
        a = dp.dp_system_create_batch(h, sys2, [inputs.MASS_CU])
        try:
            dp.dp_md_step(h, a, 23, 1.0)
            xa, va, fa = dp.dp_system_get(h, a, n)
        finally:
            dp.dp_system_destroy(a)
        b = dp.dp_system_create_batch(h, sys2, [inputs.MASS_CU])
        try:
            dp.dp_md_step(h, b, 13, 1.0)
            dp.dp_state_save(h, b, tmp_path / "batch.bin")
        finally:
            dp.dp_system_destroy(b)
        c = dp.dp_state_load(h, tmp_path / "batch.bin")
        try:
            assert dp.dp_system_step(c) == 13 and dp.lib.dp_system_batch_size(c) == 2
            dp.dp_md_step(h, c, 10, 1.0)
            xc, vc, fc = dp.dp_system_get(h, c, n)
        finally:
            dp.dp_system_destroy(c)
        assert np.array_equal(xa, xc) and np.array_equal(va, vc) and np.array_equal(fa, fc)
    finally:
        dp.dp_destroy(h)
