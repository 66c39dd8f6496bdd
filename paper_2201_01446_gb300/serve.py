"""Serving loop over the C ABI: a stream of energy/force and MD requests on
systems of mixed size, admitted under a device-memory budget and run by a
pool of worker slots, each with its own CUDA stream and its own handles (one
per model), so requests from different slots overlap on the GPU.  Results are
computed by the same deterministic kernels whatever runs beside them, so a
request's result is bitwise the one it has alone.

Small requests of one model are packed: a slot that takes a request from
the head of the queue also takes the queued requests of the same model and
kind behind it (MD requests: also the same number of steps), up to
`pack_atoms` atoms in all, and runs them as one dp_compute_batch call or one
batched MD system (one launch of each kernel for all of them; each result
still bitwise the one it has alone).  MD steps without a list rebuild replay
as a CUDA graph inside the library.

Host orchestration only (queueing, admission, timing): every step of every
request runs in the library's kernels.
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
    shape: dict = field(default_factory=dict)  # estimate_bytes: M, fit_widths


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


def estimate_bytes(natoms: int, cfg: ModelCfg, M: int = 128, fit_widths=(240, 240, 240),
                   nsys: int = 1, skin: float = 2.0) -> int:
    """Upper estimate of the device bytes a request of natoms adds to a
    trimmed handle (dp_trim) of the tensor-core modes: per atom the neighbor
    list with skin (1.5 x N_m scaled to rc + skin, + 64 entries), T and dE/dT,
    the sorted pairs of the embedding kernels (N_m + 32 per atom slot, tiles
    of 32 padded per system), bin ends and the per-atom arrays; per fitting
    row (at most 32 waves of 152 x 128 rows) the FP32 activation and gradient
    rows and the BF16 pieces of the last and the backward layers' A operands."""
    nm = int(sum(cfg.sel))
    cap = int(1.5 * nm * ((cfg.rc + skin) / cfg.rc) ** 3) + 64
    slots = natoms + 32 * nsys
    per_atom = 4 * cap + 2 * 4 * 4 * M + 400
    per_slot = 16 * ((nm + 32 + 31) // 32 * 32) + 2 * 1024  # sorted pairs, bin ends
    wmax = max(fit_widths)
    rows = min(-(-max(natoms, 1) // 128) * 128, 32 * 152 * 128)
    per_row = wmax * (4 + 3 * 2 * 3) + sum(w * (4 + 4) for w in fit_widths)
    return int(natoms * per_atom + slots * per_slot + rows * per_row + (8 << 20))


class Server:
    """Admission holds the sum of the slots' device bytes under the budget.
    A slot holds what its handles hold (measured by dp_memory after each
    request: the model, tables and the buffers kept from finished requests)
    plus, while it runs, the estimate of what its request adds.  A request
    that does not fit makes slots release their handles' kept buffers
    (dp_trim: the taking slot itself, or idle slots) before it waits; one
    larger than the budget runs alone once nothing else holds more than its
    model."""

    def __init__(self, models: dict, slots: int = 4, budget_bytes: float = 150e9,
                 pack_atoms: int = 32768):
        self.models = models
        self.slots = slots
        self.budget = float(budget_bytes)
        self.pack_atoms = int(pack_atoms)
        self.packed_calls = 0
        self.packed_requests = 0
        self._cond = threading.Condition()
        self._ready = []       # arrived, not yet admitted (FIFO)
        self._closing = False
        self._done = []
        self._held = [0.0] * slots    # bytes each slot holds (see above)
        self._fixed = [0.0] * slots   # bytes of its handles right after creation
        self._running = [False] * slots
        self._trim_req = [False] * slots
        self.trims = 0
        self.peak_in_use = 0.0

    @property
    def _in_use(self) -> float:
        return float(sum(self._held))

    # ---------------------------------------------------------------- queue
    def _push(self, req: Request) -> None:
        with self._cond:
            self._ready.append(req)
            self._cond.notify_all()

    def _take(self, k: int, can_pack: bool):
        """For slot k: the head of the queue once it fits the budget (FIFO
        admission), with, when the slot can pack and the head is small, the
        queued requests of the same model and kind (MD: same steps) behind it
        that fit; "trim" when the slot should release its kept buffers first;
        None when the server closes with nothing left."""
        with self._cond:
            while True:
                if self._trim_req[k]:
                    self._trim_req[k] = False
                    if self._held[k] > self._fixed[k]:
                        return "trim"
                if self._ready:
                    head = self._ready[0]
                    others = self._in_use - self._held[k]
                    if others + self._held[k] + head.nbytes <= self.budget:
                        return self._admit(k, head, can_pack, others)
                    if self._held[k] > self._fixed[k]:
                        return "trim"
                    idle = [j for j in range(self.slots) if j != k and not self._running[j]
                            and self._held[j] > self._fixed[j]]
                    for j in idle:
                        self._trim_req[j] = True
                    if not idle and not any(self._running):
                        return self._admit(k, head, False, others)  # larger than the budget
                    self._cond.notify_all()
                elif self._closing:
                    return None
                self._cond.wait(0.05)

    def _admit(self, k, head, can_pack, others):
        self._ready.pop(0)
        held = self._held[k] + head.nbytes
        batch = [head]
        if can_pack and len(head.x) <= self.pack_atoms:
            atoms = len(head.x)
            for r in list(self._ready):
                if (r.kind == head.kind and r.model == head.model
                        and (r.kind == "eval" or r.steps == head.steps)
                        and atoms + len(r.x) <= self.pack_atoms
                        and others + held + r.nbytes <= self.budget):
                    self._ready.remove(r)
                    held += r.nbytes
                    atoms += len(r.x)
                    batch.append(r)
        self._held[k] = held
        self._running[k] = True
        self.peak_in_use = max(self.peak_in_use, self._in_use)
        return batch

    def _finish(self, k: int, reqs: list, held_after) -> None:
        with self._cond:
            self._held[k] = self._fixed[k] if held_after is None else float(held_after)
            self._running[k] = False
            self.peak_in_use = max(self.peak_in_use, self._in_use)
            self._done.extend(reqs)
            self._cond.notify_all()

    def _set_held(self, k: int, held) -> None:
        with self._cond:
            self._held[k] = self._fixed[k] if held is None else float(held)
            self._cond.notify_all()

    # ---------------------------------------------------------------- run
    def run(self, requests: list, arrivals, executor_factory=None) -> dict:
        """Serve `requests` arriving at `arrivals` (s after the start; 0 for
        all: closed loop).  executor_factory(slot) returns a callable that
        runs one request (the default runs it through the library); an
        executor with bytes() and trim() (device bytes its handles hold,
        releasing their kept buffers) takes part in the byte accounting."""
        make = executor_factory or self._dp_executor
        execs = [make(i) for i in range(self.slots)]
        for r in requests:
            if not r.nbytes:
                cfg = self.models[r.model]
                r.nbytes = estimate_bytes(len(r.x), cfg, **getattr(cfg, "shape", {}))
        for k, ex in enumerate(execs):
            b = ex.bytes() if hasattr(ex, "bytes") else None
            self._fixed[k] = float(b or 0.0)
            self._held[k] = self._fixed[k]
            self._running[k] = False
            self._trim_req[k] = False
        self._done = []
        self._closing = False
        self.packed_calls = self.packed_requests = 0
        self.trims = 0
        self.peak_in_use = self._in_use
        t0 = time.perf_counter()

        def worker(k, ex):
            can_pack = self.pack_atoms > 0 and hasattr(ex, "batch")
            measured = hasattr(ex, "bytes")
            while True:
                reqs = self._take(k, can_pack)
                if reqs is None:
                    return
                if reqs == "trim":
                    if hasattr(ex, "trim"):
                        ex.trim()
                    with self._cond:
                        self.trims += 1
                    self._set_held(k, ex.bytes() if measured else None)
                    continue
                for r in reqs:
                    r.t_start = time.perf_counter() - t0
                try:
                    if len(reqs) == 1:
                        reqs[0].result = ex(reqs[0])
                    else:
                        for r, res in zip(reqs, ex.batch(reqs)):
                            r.result = res
                        with self._cond:
                            self.packed_calls += 1
                            self.packed_requests += len(reqs)
                except Exception as e:  # recorded, the loop goes on
                    for r in reqs:
                        r.error = str(e)
                t = time.perf_counter() - t0
                for r in reqs:
                    r.t_done = t
                self._finish(k, reqs, ex.bytes() if measured else None)

        threads = [threading.Thread(target=worker, args=(k, ex), daemon=True)
                   for k, ex in enumerate(execs)]
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
                "slots": self.slots, "peak_budget_bytes": self.peak_in_use,
                "budget_bytes": self.budget, "trims": self.trims,
                "packed_calls": self.packed_calls, "packed_requests": self.packed_requests}

    def _dp_executor(self, slot: int):
        return _DpSlot(self.models)


class _DpSlot:
    """One worker slot: its own CUDA stream and a handle per model."""

    def __init__(self, models: dict):
        import ctypes
        import torch
        self._stream = torch.cuda.Stream()
        self._sp = ctypes.c_void_p(self._stream.cuda_stream)
        self.models = models
        self.handles = {name: dp.dp_create(c.path, c.ntypes, c.rc, c.rcs, c.sel,
                                           options=c.options, stream=self._sp)
                        for name, c in models.items()}

    def batch(self, reqs: list):
        """Requests of one model and kind as one call: evaluations through
        dp_compute_batch, MD runs (same steps) as one batched system (models
        without the tensor-core tabulated embedding run them one by one)."""
        h = self.handles[reqs[0].model]
        o = self.models[reqs[0].model].options
        same_mass = all(list(r.masses) == list(reqs[0].masses) for r in reqs)
        if o is None or not (o.tabulated and o.embed_precision == 2) or not same_mass:
            return [self(r) for r in reqs]
        if reqs[0].kind == "eval":
            E, F, V = dp.dp_compute_batch(h, [(r.x, r.types, r.box) for r in reqs])
            return [(float(E[q]), F[q], V[q]) for q in range(len(reqs))]
        s = dp.dp_system_create_batch(h, [(r.x, r.v, r.types, r.box) for r in reqs],
                                      reqs[0].masses)
        try:
            dp.dp_md_step(h, s, reqs[0].steps, DT_FS[reqs[0].model])
            n = sum(len(r.x) for r in reqs)
            X, Vv, F = dp.dp_system_get(h, s, n)
        finally:
            dp.dp_system_destroy(s)
        out, o0 = [], 0
        for r in reqs:
            m = len(r.x)
            out.append((X[o0:o0 + m], Vv[o0:o0 + m], F[o0:o0 + m]))
            o0 += m
        return out

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

    def bytes(self) -> int:
        """Device bytes the slot's handles hold (dp_memory)."""
        return sum(dp.dp_memory(h)["handle"] for h in self.handles.values())

    def trim(self) -> None:
        """Release the handles' kept buffers and scratch (dp_trim)."""
        for h in self.handles.values():
            dp.dp_trim(h)

    def close(self):
        for h in self.handles.values():
            dp.dp_destroy(h)
        self.handles = {}


def make_requests(specs: list) -> list:
    """Request objects from inputs.serve_requests dicts."""
    return [Request(rid=i, model=s["model"], kind=s["kind"], x=s["x"], v=s["v"],
                    types=s["types"], box=s["box"], masses=s["masses"], steps=s["steps"])
            for i, s in enumerate(specs)]
