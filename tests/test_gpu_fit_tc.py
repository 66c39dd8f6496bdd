"""Tensor-core (tcgen05, 16-bit operands, FP32 accumulation) fitting modes.

The same per-atom descriptors go through the FP32 CUDA-core fitting stage and
the tensor-core ones; the BF16 mode's errors are measured and stated (the
paper notes that mixed precision has accuracy problems, Sec. 7), with bounds
that a wrong tile, descriptor or epilogue would exceed by orders of
magnitude.  The FP32-accurate mode (fit_precision 2: each operand three
BF16 pieces, six piece products) is held to the FP32 path's bars; the
near-FP32 mode (3: an FP16 pair under a power-of-two scale, three products)
to bars twice as wide (NEAR), its errors measured 1.2-1.5x those of mode 2:
the tensor core adds the 22-bit FP16 products of a K = 16 step with fewer
exact bits than the 16-bit BF16 ones.  Mode 4 (mode 2 with the dE/dD GEMM,
which feeds only the forces, on FP16 pairs) is held to the FP32 bars."""
import numpy as np
import pytest

import oracle
from paper_2201_01446_gb300 import inputs
from conftest import CU_RC, CU_RCS, CU_SEL, CU_SMAX, PARITY_LOG, TABLE_H, force_bar, rmse

pytestmark = pytest.mark.gpu

# bar factor of each split mode against the FP32 path's bars
NEAR = {2: 1.0, 3: 2.0, 4: 1.0}


@pytest.fixture(scope="module")
def dp():
    from paper_2201_01446_gb300 import dp as _dp
    return _dp


def _handle(dp, path, prec):
    o = dp.dp_options_default()
    o.fit_precision = prec
    return dp.dp_create(path, 1, CU_RC, CU_RCS, [CU_SEL], options=o, stream=None)


def _handles(dp, path):
    return _handle(dp, path, 0), _handle(dp, path, 1)


@pytest.mark.parametrize("std", [0.1, 1.0])
def test_tc_fitting_vs_fp32_and_oracle(dp, model_dir, std):
    path = str(model_dir / f"cu_tc_{std}.model")
    inputs.write_seeded_model(path, inputs.COPPER_SPEC, seed=0, std=std)
    h0, h1 = _handles(dp, path)
    try:
        # ragged row count (not a multiple of the 128-row tile)
        x, t, box = inputs.fcc_copper((5, 5, 6), sigma=0.1, seed=3)
        T = dp.dp_descriptor(h0, x, t, box, 128)
        e0, dT0 = dp.dp_fitting(h0, t, T)
        e1, dT1 = dp.dp_fitting(h1, t, T)
    finally:
        dp.dp_destroy(h0)
        dp.dp_destroy(h1)
    m = oracle.Model(path)
    eo = np.array([m.fit(0, np.einsum("cb,ca->ba", T[i].astype(np.float64),
                                      T[i, :, :16].astype(np.float64)).ravel())[0]
                   for i in range(0, len(x), 37)])
    de_tc = float(np.abs(e1 - e0).max())
    de_or = float(np.abs(e1[::37] - eo).max())
    ddt = float(np.abs(dT1 - dT0).max() / np.abs(dT0).max())
    PARITY_LOG.append(dict(case=f"tc bf16 fitting std {std}", natoms=len(x), max_dEi_vs_fp32=de_tc,
                           max_dEi_vs_oracle=de_or, max_rel_dT=ddt,
                           fp32_vs_oracle=float(np.abs(e0[::37] - eo).max())))
    # BF16 operands: ~2^-9 relative per operand; a broken tile, descriptor or
    # epilogue gives errors of the order of the values themselves
    scale = float(np.abs(e0).max())
    assert de_tc < 5e-2 * scale, (de_tc, scale)
    assert de_or < 5e-2 * scale
    assert ddt < 0.3, ddt
    assert np.abs(e0[::37] - eo).max() < 1e-5 * max(1, scale)


def test_tc_mode_forces_vs_oracle(dp, cu_model_path):
    # the configured model end to end with the BF16 fitting mode: errors stated
    m = oracle.Model(cu_model_path)
    tab = oracle.Table(m, TABLE_H, CU_SMAX)
    o = dp.dp_options_default()
    o.fit_precision = 1
    h = dp.dp_create(cu_model_path, 1, CU_RC, CU_RCS, [CU_SEL], options=o, stream=None)
    try:
        x, t, box = inputs.fcc_copper(5, sigma=0.05, seed=1)
        E, F, V, Ei = dp.dp_compute(h, x, t, box, atom_energy=True)
    finally:
        dp.dp_destroy(h)
    r = oracle.evaluate(m, tab, CU_RC, CU_RCS, CU_SEL, x, t, box)
    de = abs(E - r["energy"]) / len(x)
    fr = rmse(F, r["force"])
    frms = float(np.sqrt((r["force"] ** 2).mean()))
    PARITY_LOG.append(dict(case="tc bf16 config1 Cu 500", natoms=len(x), dE_per_atom=de,
                           force_rmse=fr, force_rms=frms))
    assert de < 1e-3 and fr < 0.3 * frms + 1e-9, (de, fr, frms)


@pytest.mark.parametrize("prec", [2, 3, 4])
@pytest.mark.parametrize("std", [0.1, 1.0])
def test_split_tc_fitting_matches_fp32(dp, model_dir, std, prec):
    # FP32-accurate tensor-core modes (the FP16 pair, three BF16 pieces), the
    # piece products accumulated in FP32; held to the FP32 path's error level
    path = str(model_dir / f"cu_split_{std}.model")
    inputs.write_seeded_model(path, inputs.COPPER_SPEC, seed=0, std=std)
    h0, h2 = _handle(dp, path, 0), _handle(dp, path, prec)
    try:
        x, t, box = inputs.fcc_copper((5, 5, 6), sigma=0.1, seed=3)
        T = dp.dp_descriptor(h0, x, t, box, 128)
        e0, dT0 = dp.dp_fitting(h0, t, T)
        e2, dT2 = dp.dp_fitting(h2, t, T)
    finally:
        dp.dp_destroy(h0)
        dp.dp_destroy(h2)
    m = oracle.Model(path)
    sub = list(range(0, len(x), 37))
    eo = np.array([m.fit(0, np.einsum("cb,ca->ba", T[i].astype(np.float64),
                                      T[i, :, :16].astype(np.float64)).ravel())[0] for i in sub])
    d0 = float(np.abs(e0[sub] - eo).max())
    d2 = float(np.abs(e2[sub] - eo).max())
    ddt = float(np.abs(dT2 - dT0).max() / np.abs(dT0).max())
    PARITY_LOG.append(dict(case=f"tc split fitting std {std} mode {prec}", natoms=len(x),
                           fp32_vs_oracle=d0, split_vs_oracle=d2, max_rel_dT_vs_fp32=ddt))
    # measured: about twice the FP32 CUDA-core path's error (the hi*hi
    # products and the small piece products accumulate in separate TMEM sums)
    scale = max(1.0, float(np.abs(eo).max()))
    assert d2 < 5e-6 * scale * NEAR[prec], (d2, d0)
    assert ddt < 5e-5 * NEAR[prec], ddt


@pytest.mark.parametrize("prec", [2, 3, 4])
def test_split_mode_end_to_end(dp, cu_model_path, cu_stress_path, prec):
    for path, stress in ((cu_model_path, False), (cu_stress_path, True)):
        m = oracle.Model(path)
        tab = oracle.Table(m, TABLE_H, CU_SMAX)
        h = _handle(dp, path, prec)
        try:
            x, t, box = inputs.fcc_copper(5, sigma=0.05, seed=1)
            E, F, V, Ei = dp.dp_compute(h, x, t, box, atom_energy=True)
        finally:
            dp.dp_destroy(h)
        r = oracle.evaluate(m, tab, CU_RC, CU_RCS, CU_SEL, x, t, box)
        de = abs(E - r["energy"]) / len(x)
        fr = rmse(F, r["force"])
        frms = float(np.sqrt((r["force"] ** 2).mean()))
        PARITY_LOG.append(dict(case=f"tc split mode {prec} Cu 500 stress={stress}", natoms=len(x),
                               dE_per_atom=de, force_rmse=fr, force_rms=frms))
        # the FP32 path's bars (configured: absolute; stress: FP32-relative)
        f = NEAR[prec]
        if not stress:
            assert de < 1e-6 and fr <= force_bar(frms), (de, fr, frms)
        else:
            assert de < max(1e-6, 2e-6 * f * float(np.abs(r["atom_energy"]).mean())), de
            assert fr < max(1e-5, 3e-5 * f * frms), (fr, frms)


@pytest.mark.parametrize("prec", [2, 3, 4])
def test_split_mode_water_two_types(dp, water_model_path, prec):
    # two centre types (per-type fitting nets gathered through an index list),
    # M = 100: D has 1600 columns, so the dE/dD GEMM ends in a ragged 64-column
    # tile; held to the FP32 path's stress-model bars, both errors logged
    m = oracle.Model(water_model_path)
    tab = oracle.Table(m, TABLE_H, 1.25)
    x, t, box = inputs.water_like(64, L=12.417, seed=3)
    r = oracle.evaluate(m, tab, 6.0, 0.5, [46, 92], x, t, box)
    emean = float(np.abs(r["atom_energy"]).mean())
    emax = float(np.abs(r["atom_energy"]).max())
    frms = float(np.sqrt((r["force"] ** 2).mean()))
    vmax = float(np.abs(r["virial"]).max())
    got = {}
    for pr in (0, prec):
        o = dp.dp_options_default()
        o.fit_precision = pr
        o.s_max = 1.25
        h = dp.dp_create(water_model_path, 2, 6.0, 0.5, [46, 92], options=o, stream=None)
        try:
            E, F, V, Ei = dp.dp_compute(h, x, t, box, atom_energy=True)
        finally:
            dp.dp_destroy(h)
        got[pr] = (abs(E - r["energy"]) / len(x), float(np.abs(Ei - r["atom_energy"]).max()),
                   rmse(F, r["force"]), float(np.abs(V - r["virial"]).max()))
    de, dei, fr, dv = got[prec]
    PARITY_LOG.append(dict(case=f"tc split mode {prec} water 192 std 1.0", natoms=len(x), dE_per_atom=de,
                           max_dEi=dei, force_rmse=fr, force_rms=frms, max_dvirial=dv,
                           fp32_path=dict(zip(("dE_per_atom", "max_dEi", "force_rmse",
                                               "max_dvirial"), got[0]))))
    # energies: the tensor core's FP32 accumulator adds each K = 16 step with
    # truncation, a bias that grows with K (1600 here); measured 5.6e-6 of the
    # mean |E_i| on this stress model, about twice the CUDA-core path's error
    f = NEAR[prec]
    assert de < max(1e-6, 1e-5 * f * emean), (de, emean, got[0])
    assert dei < 2e-5 * f * emax, (dei, emax)
    assert fr < max(1e-5, 3e-5 * f * frms), (fr, frms)
    assert dv < 1e-4 * f * vmax + 1e-9, (dv, vmax)


@pytest.mark.parametrize("prec", [2, 3, 4])
def test_split_mode_wide_fitting_fallback(dp, model_dir, prec):
    # fitting layers 256 wide: K = 256 is the most the persistent kernel
    # takes (16 K chunks); every K-short GEMM streams A with B through its
    # stages, the dE/dD GEMM over 16 N tiles of 128 columns
    spec = inputs.ModelSpec(1, (32, 64, 128), 16, (256, 256, 256))
    path = str(model_dir / "cu_wide256.model")
    inputs.write_seeded_model(path, spec, seed=7, std=1.0)
    m = oracle.Model(path)
    tab = oracle.Table(m, TABLE_H, CU_SMAX)
    x, t, box = inputs.fcc_copper(5, sigma=0.05, seed=1)
    r = oracle.evaluate(m, tab, CU_RC, CU_RCS, CU_SEL, x, t, box)
    o = dp.dp_options_default()
    o.fit_precision = prec
    o.embed_precision = 2
    h = dp.dp_create(path, 1, CU_RC, CU_RCS, [CU_SEL], options=o, stream=None)
    try:
        E, F, V, Ei = dp.dp_compute(h, x, t, box, atom_energy=True)
    finally:
        dp.dp_destroy(h)
    dei = float(np.abs(Ei - r["atom_energy"]).max())
    fr = rmse(F, r["force"])
    frms = float(np.sqrt((r["force"] ** 2).mean()))
    PARITY_LOG.append(dict(case=f"tc split mode {prec} Cu 500, 256-wide fitting",
                           natoms=len(x), max_dEi=dei, force_rmse=fr, force_rms=frms))
    assert dei < 2e-5 * NEAR[prec] * float(np.abs(r["atom_energy"]).max()), dei
    assert fr < max(1e-5, 3e-5 * NEAR[prec] * frms), (fr, frms)


@pytest.mark.parametrize("prec", [2, 3, 4])
@pytest.mark.parametrize("std", [1e-3, 4.0])
def test_fp16_pair_scales_follow_the_magnitudes(dp, model_dir, std, prec):
    # models whose weights, descriptors and gradients sit far outside FP16's
    # range unscaled (std 1e-3: D ~ 1e-8, below the smallest FP16 subnormal;
    # std 4: gradients in the thousands): the power-of-two scales (per row of
    # D, per weight matrix, per activation and gradient from the net's
    # bounds) keep the FP16-pair mode finite and near the FP32 path (an
    # overflowed or underflowed operand gives errors of the order of the
    # values); the BF16-triple mode beside it for comparison
    path = str(model_dir / f"cu_pair_{std}.model")
    inputs.write_seeded_model(path, inputs.COPPER_SPEC, seed=5, std=std)
    h0, h2 = _handle(dp, path, 0), _handle(dp, path, prec)
    try:
        x, t, box = inputs.fcc_copper((5, 5, 6), sigma=0.1, seed=4)
        T = dp.dp_descriptor(h0, x, t, box, 128)
        e0, dT0 = dp.dp_fitting(h0, t, T)
        e2, dT2 = dp.dp_fitting(h2, t, T)
    finally:
        dp.dp_destroy(h0)
        dp.dp_destroy(h2)
    m = oracle.Model(path)
    sub = list(range(0, len(x), 37))
    eo = np.array([m.fit(0, np.einsum("cb,ca->ba", T[i].astype(np.float64),
                                      T[i, :, :16].astype(np.float64)).ravel())[0] for i in sub])
    assert np.all(np.isfinite(e2)) and np.all(np.isfinite(dT2))
    d0 = float(np.abs(e0[sub] - eo).max())
    d2 = float(np.abs(e2[sub] - eo).max())
    ddt = float(np.abs(dT2 - dT0).max() / max(float(np.abs(dT0).max()), 1e-30))
    PARITY_LOG.append(dict(case=f"tc split mode {prec} fitting std {std}", natoms=len(x),
                           fp32_vs_oracle=d0, pair_vs_oracle=d2, max_rel_dT_vs_fp32=ddt,
                           max_abs_T=float(np.abs(T).max()), max_abs_dT=float(np.abs(dT0).max())))
    scale = float(np.abs(eo).max())
    assert d2 < 1e-4 * scale + 1e-12, (d2, d0, scale)
    assert ddt < 5e-3, ddt


@pytest.mark.parametrize("prec", [2, 4])
@pytest.mark.parametrize("fit_w", [(240, 240), (240, 160, 160, 160), (128, 240, 240)])
def test_split_mode_fitting_shapes(dp, model_dir, fit_w, prec):
    # fitting nets other than three 240-wide layers: two layers (layer 0 writes
    # the last layer's pieces itself), two hidden layers with a width change
    # (no shortcut there, a shortcut after), a narrow layer 0 (N = 128) below
    # wider ones; end to end against the oracle, beside the FP32 CUDA-core path
    # on the same inputs
    spec = inputs.ModelSpec(1, (32, 64, 128), 16, fit_w)
    path = str(model_dir / f"cu_fit_{'_'.join(map(str, fit_w))}.model")
    inputs.write_seeded_model(path, spec, seed=11, std=1.0)
    m = oracle.Model(path)
    tab = oracle.Table(m, TABLE_H, CU_SMAX)
    x, t, box = inputs.fcc_copper((4, 5, 5), sigma=0.1, seed=6)
    r = oracle.evaluate(m, tab, CU_RC, CU_RCS, CU_SEL, x, t, box)
    err = {}
    for pr in (0, prec):
        o = dp.dp_options_default()
        o.fit_precision = pr
        o.embed_precision = 2 if pr else 0
        h = dp.dp_create(path, 1, CU_RC, CU_RCS, [CU_SEL], options=o, stream=None)
        try:
            E, F, V, Ei = dp.dp_compute(h, x, t, box, atom_energy=True)
        finally:
            dp.dp_destroy(h)
        assert np.isfinite(E) and np.all(np.isfinite(F))
        err[pr] = (abs(E - r["energy"]) / len(x), float(np.abs(Ei - r["atom_energy"]).max()),
                   rmse(F, r["force"]), float(np.abs(V - r["virial"]).max()))
    emean = float(np.abs(r["atom_energy"]).mean())
    emax = float(np.abs(r["atom_energy"]).max())
    frms = float(np.sqrt((r["force"] ** 2).mean()))
    vmax = float(np.abs(r["virial"]).max())
    de, dei, fr, dv = err[prec]
    PARITY_LOG.append(dict(case=f"tc split mode {prec} Cu {len(x)} fitting {fit_w}",
                           natoms=len(x), dE_per_atom=de, max_dEi=dei, force_rmse=fr,
                           force_rms=frms, max_dvirial=dv, mean_abs_Ei=emean,
                           fp32_path=dict(zip(("dE_per_atom", "max_dEi", "force_rmse",
                                               "max_dvirial"), err[0]))))
    # these shapes test the kernels' shape handling (ragged N tiles, K chunk
    # counts, layers without a shortcut, layer 0 writing the last layer's
    # pieces): a mis-tiled operand or a skipped term gives errors of the order
    # of the values.  The accuracy bars proper are those of the configured
    # shapes; on these nets the split modes measured up to 2.4x the FP32
    # CUDA-core path's force error and 9x its total-energy error (the tensor
    # core's accumulation bias, which depends on the net), so the bound is
    # the stress-model bars or a few times the FP32 path's own error
    f0 = err[0]
    assert de < max(1e-6, 5e-6 * emean, 12 * f0[0]), (de, emean, f0)
    assert dei < max(2e-5 * emax, 3 * f0[1]), (dei, emax, f0)
    assert fr < max(1e-5, 3e-5 * frms, 3 * f0[2]), (fr, frms, f0)
    assert dv < max(1e-4 * vmax + 1e-9, 15 * f0[3]), (dv, vmax, f0)
