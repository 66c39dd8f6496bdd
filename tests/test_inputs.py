"""The synthetic inputs' recipes (CPU): the bench's water leg replicates the
seeded water box, which must be the periodic extension of the original, so
the FP64 oracle gives every copy the original's energies and forces (the
model's extensivity under periodic replication)."""
import numpy as np

import oracle
from paper_2201_01446_gb300 import inputs
from conftest import TABLE_H


def test_replicated_water_box_is_its_periodic_extension(water_model_path):
    x0, t0, box0 = inputs.water_like(64, L=12.417, seed=3)
    x, t, box = inputs.replicate(x0, t0, box0, 2)
    assert len(x) == 8 * len(x0) and np.allclose(np.diag(box), 2 * np.diag(box0))
    # no pair closer than the packing allows (O-H 0.96 A is the closest)
    assert len(oracle.neighbors(x, box, 0.9)) == 0
    m = oracle.Model(water_model_path)
    tab = oracle.Table(m, TABLE_H, 1.25)
    r0 = oracle.evaluate(m, tab, 6.0, 0.5, [46, 92], x0, t0, box0)
    r = oracle.evaluate(m, tab, 6.0, 0.5, [46, 92], x, t, box)
    n0 = len(x0)
    for c in range(8):
        sl = slice(c * n0, (c + 1) * n0)
        assert np.allclose(r["atom_energy"][sl], r0["atom_energy"], rtol=0, atol=1e-10)
        assert np.allclose(r["force"][sl], r0["force"], rtol=0, atol=1e-9)
    assert abs(r["energy"] - 8 * r0["energy"]) < 1e-8 * abs(r0["energy"]) * 8 + 1e-9
