"""Serving loop on the GPU: a mixed request stream (copper and water boxes,
evaluations and MD runs) through three concurrent slots gives, request by
request, bitwise the results of the same request run alone on a fresh
handle."""
import numpy as np
import pytest

from paper_2201_01446_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_results_bitwise_alone_and_in_the_mix(cu_model_path, model_dir):
    from paper_2201_01446_gb300 import dp, serve
    wpath = str(model_dir / "water_serve.model")
    inputs.write_seeded_model(wpath, inputs.WATER_SPEC, seed=4, std=0.1)

    def opts(s_max):
        # the bench's modes (the split-BF16 mode 2 is covered packed and alone
        # by the batch tests)
        o = dp.dp_options_default()
        o.fit_precision = 4
        o.embed_precision = 2
        o.s_max = s_max
        return o

    models = {"cu": serve.ModelCfg(cu_model_path, 1, 8.0, 0.5, [256], opts(2.0)),
              "water": serve.ModelCfg(wpath, 2, 6.0, 0.5, [46, 92], opts(2.0))}
    specs = inputs.serve_requests(12, seed=9, max_atoms=20000, md_steps=12)
    reqs = serve.make_requests(specs)
    srv = serve.Server(models, slots=3)
    st = srv.run(reqs, inputs.poisson_arrivals(len(reqs), 200.0, seed=2))
    assert st["errors"] == 0, [r.error for r in reqs if r.error]
    alone = serve._DpSlot(models)
    try:
        for r in serve.make_requests(specs):
            ref = alone(r)
            got = reqs[r.rid].result
            for a, b in zip(got, ref):
                assert np.array_equal(np.asarray(a), np.asarray(b)), (r.rid, r.model, r.kind)
    finally:
        alone.close()
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_device_bytes_stay_under_the_budget(cu_model_path, model_dir):
    # a 2 GB budget against a stream whose requests (copper up to 40,000
    # atoms, water up to 24,576) each need a few hundred MB: what the
    # library really allocated (its own byte counter, every cudaMalloc and
    # cudaFree) never passes the budget, kept buffers are released for the
    # larger requests, and every request is served
    from paper_2201_01446_gb300 import dp, serve
    wpath = str(model_dir / "water_budget.model")
    inputs.write_seeded_model(wpath, inputs.WATER_SPEC, seed=4, std=0.1)

    def opts():
        o = dp.dp_options_default()
        o.fit_precision = 2
        o.embed_precision = 2
        return o

    models = {"cu": serve.ModelCfg(cu_model_path, 1, 8.0, 0.5, [256], opts()),
              "water": serve.ModelCfg(wpath, 2, 6.0, 0.5, [46, 92], opts(), {"M": 100})}
    specs = inputs.serve_requests(24, seed=13, max_atoms=40000, md_steps=10, water_md_steps=10)
    reqs = serve.make_requests(specs)
    budget = 2e9
    base = dp.dp_memory(reset_peak=True)["process"]
    srv = serve.Server(models, slots=3, budget_bytes=budget)
    st = srv.run(reqs, inputs.poisson_arrivals(len(reqs), 100.0, seed=3))
    mem = dp.dp_memory()
    assert st["errors"] == 0, [r.error for r in reqs if r.error]
    assert all(r.result is not None for r in reqs)
    assert srv.peak_in_use <= budget
    assert mem["peak"] - base <= budget, (mem["peak"] - base, budget)
    assert st["trims"] > 0
    # the slots' handles are destroyed: nothing of theirs is held any more
    assert mem["process"] == base
