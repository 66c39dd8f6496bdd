"""The energy as a torch.autograd function of the positions: its gradient is
the library's -F (bitwise), and gradients compose through torch ops."""
import numpy as np
import pytest

from paper_2201_01446_gb300 import inputs
from conftest import CU_RC, CU_RCS, CU_SEL

pytestmark = pytest.mark.gpu


def test_energy_gradient_is_minus_forces(cu_stress_path):
    torch = pytest.importorskip("torch")
    from paper_2201_01446_gb300 import autograd, dp
    o = dp.dp_options_default()
    o.fit_precision = 2
    o.embed_precision = 2
    h = dp.dp_create(cu_stress_path, 1, CU_RC, CU_RCS, [CU_SEL], options=o)
    try:
        xn, tn, bn = inputs.fcc_copper(5, sigma=0.05, seed=1)
        x = torch.tensor(xn, device="cuda", requires_grad=True)
        t = torch.tensor(tn, device="cuda")
        box = torch.tensor(bn, device="cuda")
        E, V, Ei = autograd.energy(h, x, t, box)
        (gx,) = torch.autograd.grad(E, x)
        E2, F, V2, _ = dp.dp_compute(h, torch.tensor(xn, device="cuda"), t, box)
        torch.cuda.synchronize()
        assert float(E.detach()) == float(E2[0])
        assert torch.equal(gx, -F) and torch.equal(V, V2)
        assert abs(float(Ei.sum()) - float(E.detach())) < 1e-9 * abs(float(E.detach()))
        # composition: L = 2 E + sum(x^2)  ->  dL/dx = -2 F + 2 x
        E, _, _ = autograd.energy(h, x, t, box)
        loss = 2.0 * E + (x * x).sum()
        loss.backward()
        assert torch.allclose(x.grad, -2.0 * F + 2.0 * x.detach(), rtol=0, atol=1e-12)
        # sum of forces vanishes (translation invariance) through the gradient
        # too, to the FP32 rounding of the per-atom pair sums
        assert float(gx.sum(0).abs().max()) < 3e-5 * float(gx.abs().max())
    finally:
        dp.dp_destroy(h)
