"""Tensor-core tabulated embedding (embed_precision 2): the contraction of the
interval-grouped environment matrix with the table on tcgen05 with FP32-
accurate split operands.  Held to the same bars as the FP32 CUDA-core path
against the FP64 oracle, on the configured model, the stress model, two
centre types, ragged tiles and the degenerate cases."""
import numpy as np
import pytest

import oracle
from paper_2201_01446_gb300 import inputs
from conftest import CU_RC, CU_RCS, CU_SEL, CU_SMAX, TABLE_H
from test_gpu_parity import _parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    from paper_2201_01446_gb300 import dp as _dp
    return _dp


def _handle(dp, path, ntypes=1, rc=CU_RC, rcs=CU_RCS, sel=(CU_SEL,), **opt):
    o = dp.dp_options_default()
    o.embed_precision = 2
    o.fit_precision = 2
    for k, v in opt.items():
        setattr(o, k, v)
    return dp.dp_create(path, ntypes, rc, rcs, list(sel), options=o, stream=None)


@pytest.fixture(scope="module")
def cu_tc(dp, cu_stress_path):
    h = _handle(dp, cu_stress_path)
    m = oracle.Model(cu_stress_path)
    yield h, m, oracle.Table(m, TABLE_H, CU_SMAX)
    dp.dp_destroy(h)


def test_descriptor_tc_matches_oracle_and_fp32(dp, cu_tc, cu_stress_path):
    h, m, tab = cu_tc
    # 500 atoms: 15 full tiles and a ragged one of 20
    x, t, box = inputs.fcc_copper(5, sigma=0.05, seed=1)
    T2 = dp.dp_descriptor(h, x, t, box, m.M)
    h0 = dp.dp_create(cu_stress_path, 1, CU_RC, CU_RCS, [CU_SEL], options=None, stream=None)
    try:
        T0 = dp.dp_descriptor(h0, x, t, box, m.M)
    finally:
        dp.dp_destroy(h0)
    scale = np.abs(T0).max()
    assert np.abs(T2 - T0).max() < 2e-6 * scale
    for i in [0, 31, 32, 250, 499]:
        Tref, _ = oracle.atom_descriptor(m, tab, CU_RC, CU_RCS, CU_SEL, x, t, box, i)
        err = np.abs(T2[i] - Tref).max()
        assert err < 2e-6 * np.abs(Tref).max(), (i, err)


def test_config1_parity_tc(dp, cu_model_path):
    h = _handle(dp, cu_model_path)
    try:
        m = oracle.Model(cu_model_path)
        x, t, box = inputs.fcc_copper(5, sigma=0.05, seed=1)
        _parity(dp, h, m, oracle.Table(m, TABLE_H, CU_SMAX), x, t, box, tag="tc-embed config1 Cu 500")
    finally:
        dp.dp_destroy(h)


@pytest.mark.parametrize("ncell,sigma", [(5, 0.05), ((3, 4, 5), 0.15), (7, 0.1)])
def test_stress_parity_tc(dp, cu_tc, ncell, sigma):
    h, m, tab = cu_tc
    x, t, box = inputs.fcc_copper(ncell, sigma=sigma, seed=2)
    # the total energy carries the tensor core's accumulation bias (each K = 16
    # step is added to the FP32 accumulator with truncation): measured 2.2e-6
    # of the mean |E_i| on this stress model, the FP32 CUDA-core bar is 2e-6
    _parity(dp, h, m, tab, x, t, box, stress=True, tag=f"tc-embed stress Cu {ncell} {sigma}",
            e_rel=5e-6)


@pytest.mark.parametrize("ncell,sigma", [(5, 0.05), ((3, 4, 5), 0.15), (7, 0.1)])
def test_stress_parity_tc_pair_dedd(dp, cu_stress_path, ncell, sigma):
    # fit_precision 4: the dE/dD GEMM (forces only) on FP16 pairs, the same bars
    h = _handle(dp, cu_stress_path, fit_precision=4)
    try:
        m = oracle.Model(cu_stress_path)
        tab = oracle.Table(m, TABLE_H, CU_SMAX)
        x, t, box = inputs.fcc_copper(ncell, sigma=sigma, seed=2)
        _parity(dp, h, m, tab, x, t, box, stress=True,
                tag=f"tc-embed fit 4 stress Cu {ncell} {sigma}", e_rel=5e-6)
    finally:
        dp.dp_destroy(h)


def test_water_two_types_tc(dp, water_model_path):
    # two centre types: type-grouped tiles, each with its own table; M = 100
    # (MMA N = 112, padded columns).  Energy bar as for the tensor-core fitting
    # on this model (its K = 1600 layer-0 sums dominate the accumulation bias)
    m = oracle.Model(water_model_path)
    tab = oracle.Table(m, TABLE_H, 1.25)
    h = _handle(dp, water_model_path, ntypes=2, rc=6.0, rcs=0.5, sel=(46, 92), s_max=1.25)
    try:
        x, t, box = inputs.water_like(64, L=12.417, seed=3)
        _parity(dp, h, m, tab, x, t, box, sel=[46, 92], rc=6.0, rcs=0.5, stress=True,
                tag="tc-embed water 192 std 1.0", e_rel=1e-5)
    finally:
        dp.dp_destroy(h)


def test_edge_cases_tc(dp, cu_tc):
    h, m, tab = cu_tc
    box = np.diag([40.0, 40.0, 40.0])
    E, F, V, _ = dp.dp_compute(h, np.zeros((0, 3)), np.zeros(0, np.int32), box)
    assert E == 0.0 and F.shape == (0, 3)
    # one atom: a tile with no pair at all (no MMA), E = fitting net at D = 0
    E, F, V, _ = dp.dp_compute(h, np.array([[1.0, 2.0, 3.0]]), np.zeros(1, np.int32), box)
    E0, _ = m.fit(0, np.zeros(m.din))
    assert abs(E - E0) < 1e-5 * max(1.0, abs(E0)) and np.all(F == 0)
    # isolated atoms next to a dimer and a close contact
    x = np.array([[10, 10, 10], [12.5, 10.3, 9.8], [30, 30, 30], [5, 30, 12], [5.2, 31.3, 12.4]],
                 float)
    _parity(dp, h, m, tab, x, np.zeros(len(x), np.int32), box, stress=True,
            tag="tc-embed sparse 5 atoms", e_rel=5e-6)


def test_sel_overflow_tc(dp, cu_stress_path):
    h = _handle(dp, cu_stress_path, sel=(100,))
    try:
        x, t, box = inputs.fcc_copper(4, sigma=0.0)
        with pytest.raises(dp.DPError) as e:
            dp.dp_compute(h, x, t, box)
        assert e.value.code == 5
    finally:
        dp.dp_destroy(h)


def test_bitwise_reproducible_tc(dp, cu_tc):
    h, _, _ = cu_tc
    x, t, box = inputs.fcc_copper(6, sigma=0.1, seed=4)
    a = dp.dp_compute(h, x, t, box, atom_energy=True)
    b = dp.dp_compute(h, x, t, box, atom_energy=True)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[3], b[3])
