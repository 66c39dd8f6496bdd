"""The Sec. 3.5 tanh table in the fitting net (tanh_table = 1), on the CUDA-core
and the tensor-core fitting paths, against the oracle evaluating the same
table; and the table's effect on the energy against exact tanh (stated)."""
import numpy as np
import pytest

import oracle
from paper_2201_01446_gb300 import inputs
from conftest import CU_RC, CU_RCS, CU_SEL, CU_SMAX, PARITY_LOG, TABLE_H
from test_gpu_parity import _parity

pytestmark = pytest.mark.gpu


@pytest.fixture
def table_mode():
    oracle.set_tanh_table(True)
    yield
    oracle.set_tanh_table(False)


def _h(dp, path, fit, embed, table):
    o = dp.dp_options_default()
    o.fit_precision = fit
    o.embed_precision = embed
    o.tanh_table = table
    return dp.dp_create(path, 1, CU_RC, CU_RCS, [CU_SEL], options=o, stream=None)


@pytest.mark.parametrize("fit,embed", [(0, 0), (2, 2)])
def test_tanh_table_parity(cu_model_path, cu_stress_path, table_mode, fit, embed):
    from paper_2201_01446_gb300 import dp
    for path, stress in ((cu_model_path, False), (cu_stress_path, True)):
        m = oracle.Model(path)
        tab = oracle.Table(m, TABLE_H, CU_SMAX)
        h = _h(dp, path, fit, embed, 1)
        try:
            x, t, box = inputs.fcc_copper(5, sigma=0.05, seed=1)
            _parity(dp, h, m, tab, x, t, box, stress=stress,
                    tag=f"tanh table fit {fit} embed {embed} stress={stress}",
                    e_rel=2e-6 if fit == 0 else 5e-6)
        finally:
            dp.dp_destroy(h)


def test_tanh_table_vs_exact_stated(cu_model_path):
    from paper_2201_01446_gb300 import dp
    x, t, box = inputs.fcc_copper(5, sigma=0.05, seed=1)
    out = {}
    for table in (0, 1):
        h = _h(dp, cu_model_path, 2, 2, table)
        try:
            out[table] = dp.dp_compute(h, x, t, box, atom_energy=True)
        finally:
            dp.dp_destroy(h)
    de = float(np.abs(out[1][3] - out[0][3]).max())
    df = float(np.sqrt(((out[1][1] - out[0][1]) ** 2).mean()))
    PARITY_LOG.append(dict(case="tanh table vs exact tanh, Cu 500 configured", natoms=len(x),
                           max_dEi=de, force_rmse=df,
                           force_rms=float(np.sqrt((out[0][1] ** 2).mean()))))
    # table error < 2.3e-7 per activation, 720 activations per atom
    assert de < 1e-4 and df < 1e-6
