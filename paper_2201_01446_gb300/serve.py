"""Serving loop over the C ABI: a stream of energy/force and MD requests on
systems of mixed size, admitted under a device-memory budget and run by a
pool of worker slots, each with its own CUDA stream and its own handles (one
per model), so requests from different slots overlap on the GPU.  Results are
computed by the same deterministic kernels whatever runs beside them, so a
request's result is bitwise the one it has alone.

Host orchestration only (queueing, admission, timing): every step of every
request runs in the library's kernels.  Packing several small systems into
one ragged launch and CUDA graphs per size bucket are not built: small
requests overlap through the slots' streams instead.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import dp

DT_FS = {"cu": 1.0, "water": 0.5}


@dataclass
class ModelCfg:
    """One model the server can run: file and the dp_create arguments."""
    path: str
    ntypes: int
    rc: float
    rcs: float
    sel: list
    options: object = None


@dataclass
class Request:
    rid: int
    model: str
    kind: str            # "eval" (energy, forces, virial) or "md" (steps of velocity-Verlet)
    x: np.ndarray
    v: np.ndarray
    types: np.ndarray
    box: np.ndarray
    masses: list
    steps: int = 0
    arrival: float = 0.0
    nbytes: int = 0
    t_start: float = 0.0
    t_done: float = 0.0
    result: tuple = field(default=None, repr=False)
    error: str = ""

    @property
    def atom_steps(self) -> int:
        return len(self.x) * (self.steps if self.kind == "md" else 1)


def estimate_bytes(natoms: int, cfg: ModelCfg, M: int = 128) -> int:
    """Device bytes a request of natoms holds while it runs: neighbor list
    (about 1.25 x the pairs within rc + skin, + 32), T and dE/dT, the sorted
    pairs of the tensor-core embedding, positions, velocities, forces."""
    nm = int(sum(cfg.sel))
    cap = int(1.25 * nm * ((cfg.rc + 2.0) / cfg.rc) ** 3) + 32
    per_atom = 4 * cap + 2 * 4 * 4 * M + 16 * (nm + 64) + 256
    return natoms * per_atom + (64 << 20)


class Server:
    def __init__(self, models: dict, slots: int = 4, budget_bytes: float = 150e9):
        self.models = models
        self.slots = slots
        self.budget = float(budget_bytes)
        self._cond = threading.Condition()
        self._ready = []       # arrived, not yet admitted (FIFO)
        self._in_use = 0.0
        self._closing = False
        self._done = []
        self.peak_in_use = 0.0

    # ---------------------------------------------------------------- queue
    def _push(self, req: Request) -> None:
        with self._cond:
            self._ready.append(req)
            self._cond.notify_all()

    def _take(self):
        """Head of the queue once it fits the budget (FIFO admission); None
        when the server closes with nothing left."""
        with self._cond:
            while True:
                if self._ready:
                    head = self._ready[0]
                    if self._in_use + head.nbytes <= self.budget or self._in_use == 0.0:
                        self._ready.pop(0)
                        self._in_use += head.nbytes
                        self.peak_in_use = max(self.peak_in_use, self._in_use)
                        return head
                elif self._closing:
                    return None
                self._cond.wait(0.05)

    def _finish(self, req: Request) -> None:
        with self._cond:
            self._in_use -= req.nbytes
            self._done.append(req)
            self._cond.notify_all()

    # ---------------------------------------------------------------- run
    def run(self, requests: list, arrivals, executor_factory=None) -> dict:
        """Serve `requests` arriving at `arrivals` (s after the start; 0 for
        all: closed loop).  executor_factory(slot) returns a callable that
        runs one request (the default runs it through the library)."""
        for r in requests:
            r.nbytes = r.nbytes or estimate_bytes(len(r.x), self.models[r.model])
        make = executor_factory or self._dp_executor
        execs = [make(i) for i in range(self.slots)]
        self._done = []
        self._closing = False
        t0 = time.perf_counter()

        def worker(ex):
            while True:
                req = self._take()
                if req is None:
                    return
                req.t_start = time.perf_counter() - t0
                try:
                    req.result = ex(req)
                except Exception as e:  # recorded, the loop goes on
                    req.error = str(e)
                req.t_done = time.perf_counter() - t0
                self._finish(req)

        threads = [threading.Thread(target=worker, args=(ex,), daemon=True) for ex in execs]
        for th in threads:
            th.start()
        order = np.argsort(np.asarray(arrivals, np.float64), kind="stable")
        for i in order:
            r = requests[i]
            r.arrival = float(arrivals[i])
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            self._push(r)
        with self._cond:
            self._closing = True
            self._cond.notify_all()
        for th in threads:
            th.join()
        makespan = max(r.t_done for r in requests) if requests else 0.0
        for ex in execs:
            close = getattr(ex, "close", None)
            if close:
                close()
        lat = np.array([(r.t_done - r.arrival) * 1e3 for r in requests])
        return {"requests": len(requests), "errors": sum(bool(r.error) for r in requests),
                "makespan_s": makespan,
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else 0.0,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else 0.0,
                "atom_steps_per_s": sum(r.atom_steps for r in requests) / max(makespan, 1e-9),
                "slots": self.slots, "peak_budget_bytes": self.peak_in_use}

    def _dp_executor(self, slot: int):
        return _DpSlot(self.models)


class _DpSlot:
    """One worker slot: its own CUDA stream and a handle per model."""

    def __init__(self, models: dict):
        import ctypes
        import torch
        self._stream = torch.cuda.Stream()
        self._sp = ctypes.c_void_p(self._stream.cuda_stream)
        self.handles = {name: dp.dp_create(c.path, c.ntypes, c.rc, c.rcs, c.sel,
                                           options=c.options, stream=self._sp)
                        for name, c in models.items()}

    def __call__(self, req: Request):
        h = self.handles[req.model]
        if req.kind == "eval":
            E, F, V, _ = dp.dp_compute(h, req.x, req.types, req.box)
            return (E, F, V)
        s = dp.dp_system_create(h, req.x, req.v, req.types, req.masses, req.box)
        try:
            dp.dp_md_step(h, s, req.steps, DT_FS[req.model])
            return dp.dp_system_get(h, s, len(req.x))
        finally:
            dp.dp_system_destroy(s)

    def close(self):
        for h in self.handles.values():
            dp.dp_destroy(h)
        self.handles = {}


def make_requests(specs: list) -> list:
    """Request objects from inputs.serve_requests dicts."""
    return [Request(rid=i, model=s["model"], kind=s["kind"], x=s["x"], v=s["v"],
                    types=s["types"], box=s["box"], masses=s["masses"], steps=s["steps"])
            for i, s in enumerate(specs)]
