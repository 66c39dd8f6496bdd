"""The bench's roofline bookkeeping on CPU: the algorithmic FLOPs per unit
and the piece products per multiply-add of each fitting mode, derived here
from the layer shapes of the models (Sec. 2.1 fitting net, Sec. 3.2 quintic
table), not from the bench's own formulas."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def fitting_macs(din, widths):
    """Multiply-adds of one fitting-net pass per atom: every layer's
    in x out, then the linear output layer (width -> 1)."""
    shapes = list(zip([din] + widths[:-1], widths)) + [(widths[-1], 1)]
    return sum(a * b for a, b in shapes)


@pytest.mark.parametrize("M,din", [(128, 2048), (100, 1600)])
def test_flops_per_unit_from_layer_shapes(M, din):
    u = bench.flops_per_unit(M=M, din=din)
    # forward per pair and column: value of the quintic by Horner (5 FMA) and
    # its outer product with the four components of R (4 FMA)
    assert u["embed_contract_fwd"] == ("pair", 2 * (5 + 4) * M)
    # backward per pair and column: value and slope of the quintic (5 + 4
    # FMA), dE/dR (4) and dE/ds (5 through the 4 components and the slope)
    assert u["embed_contract_bwd_forces"] == ("pair", 2 * (5 + 4 + 4 + 5) * M)
    # fitting: the forward pass and the input gradient (the same shapes)
    assert u["fitting"] == ("atom", 2 * 2 * fitting_macs(din, [240, 240, 240]))


def test_piece_products_per_mode():
    assert bench.fit_products(0) == 1 and bench.fit_products(1) == 1
    assert bench.fit_products(2) == 6 and bench.fit_products(3) == 3
    # mode 4: six products everywhere except the dE/dD GEMM (din x 240
    # multiply-adds per atom, three FP16-pair products)
    for din in (2048, 1600):
        tot = 2 * fitting_macs(din, [240, 240, 240])
        dd = din * 240
        want = (6 * (tot - dd) + 3 * dd) / tot
        assert bench.fit_products(4, din=din) == pytest.approx(want, rel=1e-12)
    assert 4.7 < bench.fit_products(4) < 4.8
