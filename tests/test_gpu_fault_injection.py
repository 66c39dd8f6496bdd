"""Failure detection with a host-side injected fault: DP_FAULT=alloc:N makes
the N-th device allocation of the process report an out-of-memory error
(nothing on the GPU is disturbed).  Wherever that allocation falls -- in
dp_create, in the first evaluation's buffers, lists or fitting scratch --
the call must return DP_ERR_OOM, the handle must stay usable, and the
retried call must give bitwise the result of a run without the fault.
Each N runs in a child process (the injection point is read once per
process); N grows until a run meets no fault, i.e. every allocation site of
the sequence has been made to fail once."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

CHILD = r"""
import hashlib, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2201_01446_gb300 import dp, inputs
path, prec = sys.argv[2], int(sys.argv[3])
events = []
def retry(what, fn):
    for _ in range(3):
        try:
            return fn()
        except dp.DPError as e:
            events.append([what, e.code])
    raise SystemExit("no recovery after 3 tries")
o = dp.dp_options_default()
o.fit_precision = prec
o.embed_precision = prec
h = retry("create", lambda: dp.dp_create(path, 1, 8.0, 0.5, [256], options=o, stream=None))
x, t, box = inputs.fcc_copper(4, sigma=0.05, seed=3)
E, F, V = retry("compute", lambda: dp.dp_compute(h, x, t, box))[:3]
v = inputs.maxwell_velocities(np.full(len(x), inputs.MASS_CU), 330.0, seed=2)
s = retry("system", lambda: dp.dp_system_create(h, x, v, t, [inputs.MASS_CU], box))
retry("md", lambda: dp.dp_md_step(h, s, 12, 1.0))
xg = dp.dp_system_get(h, s, len(x))[0]
dp.dp_system_destroy(s)
dp.dp_destroy(h)
dig = hashlib.sha256(np.float64(E).tobytes() + F.tobytes() + V.tobytes() + xg.tobytes()).hexdigest()
print(json.dumps({"events": events, "digest": dig}))
"""


def _run(path, prec, fault):
    env = dict(os.environ, DP_SKIP_BUILD="1")
    env.pop("DP_FAULT", None)
    if fault:
        env["DP_FAULT"] = f"alloc:{fault}"
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, path, str(prec)], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (fault, r.stdout[-2000:], r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("prec", [0, 2])
def test_injected_allocation_failure_recovers(cu_stress_path, prec):
    from paper_2201_01446_gb300 import dp  # noqa: F401  (builds the library first)
    ref = _run(cu_stress_path, prec, 0)
    assert ref["events"] == []
    where = set()
    for n in range(1, 200):
        got = _run(cu_stress_path, prec, n)
        if not got["events"]:
            break
        # one injected failure: one DP_ERR_OOM, then a clean retry with the
        # result of the run without the fault
        assert got["events"] == [[got["events"][0][0], 4]], (n, got["events"])
        assert got["digest"] == ref["digest"], n
        where.add(got["events"][0][0])
    else:
        raise AssertionError("every run met a fault")
    assert n > 1 and {"create", "compute", "system"} <= where, (n, where)


WAIT_CHILD = r"""
import hashlib, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2201_01446_gb300 import dp, inputs
path = sys.argv[2]
o = dp.dp_options_default()
o.fit_precision = 2
o.embed_precision = 2
h = dp.dp_create(path, 1, 8.0, 0.5, [256], options=o, stream=None)
x, t, box = inputs.fcc_copper(5, sigma=0.05, seed=1)
codes = []
for _ in range(2):
    try:
        E, F, V, _ = dp.dp_compute(h, x, t, box)
        codes.append(0)
    except dp.DPError as e:
        codes.append(e.code)
        msg = str(e)
dig = hashlib.sha256(np.float64(E).tobytes() + F.tobytes() + V.tobytes()).hexdigest()
dp.dp_destroy(h)
print(json.dumps({"codes": codes, "digest": dig}))
"""


def test_device_wait_timeout_reports_and_recovers(cu_stress_path):
    # DP_FAULT=wait:1: the first launch of the tensor-core embedding forward
    # gives its generator warps' wait on the MMAs zero polls, so the wait
    # runs out on the device (no fault, no hang: the CTA raises its abort
    # flag, drains its own copies and MMAs with the full limit, frees its
    # TMEM and records the timeout).  The call reports DP_ERR_TIMEOUT; the
    # next call on the same handle gives the result of a run without it.
    from paper_2201_01446_gb300 import dp  # noqa: F401  (builds the library first)
    env = dict(os.environ, DP_SKIP_BUILD="1")
    env.pop("DP_FAULT", None)
    runs = {}
    for fault in ("", "wait:1"):
        e = dict(env, DP_FAULT=fault) if fault else env
        r = subprocess.run([sys.executable, "-c", WAIT_CHILD, ROOT, cu_stress_path], env=e,
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, (fault, r.stdout[-2000:], r.stderr[-2000:])
        runs[fault] = json.loads(r.stdout.strip().splitlines()[-1])
    assert runs[""]["codes"] == [0, 0]
    assert runs["wait:1"]["codes"] == [8, 0]
    assert runs["wait:1"]["digest"] == runs[""]["digest"]
