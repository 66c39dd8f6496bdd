#!/usr/bin/env python
"""Benchmark: compressed DP-SE_a copper MD on GB300, atom-steps/s per GPU.

Workload: FCC copper 100x100x100 cells (4,000,000 atoms, a = 3.634 A,
periodic), 330 K Maxwell velocities, the seeded N(0, 0.1) model of the paper's
shape (embedding 1-32-64-128, M^< = 16, fitting 2048-240-240-240-1, rc 8 A,
rcs 0.5 A, sel 256), tabulated embedding (h = 0.01) fused with the
contraction, FP32-accurate tensor-core modes for the contraction and the
fitting net, velocity-Verlet at dt = 1 fs, list rebuild every 10
steps with a 2 A skin.  One bench step is one 10-MD-step block (one list
rebuild and 10 force evaluations), so the default 10 steps are the 100 MD
steps of the workload.  No system runs past those 100 MD steps: more bench
steps run on fresh systems from the same initial state, each created (list
build and first force evaluation) outside the CUDA-event windows, whose
times are summed; warm-up runs on systems of its own.  Inputs (T, dT,
lists, sorted pairs: ~50 GB) are far larger than L2.

JSON line fields beyond the base contract: roofline (dominant phase, live
CUDA-event time), cpu_baseline (the FP64 oracle on a bounded sample of the
same configuration, also giving the sampled force/energy error), e2e
(through dp_system_create / dp_md_step / dp_system_get with host buffers),
clocks (nvidia-smi sampled during the timed region); beside the headline:
plain (the untabulated comparator), serve (the request loop), param_grad,
water (MD of a replicated two-type water-like box).

--impl reference runs the FP64 oracle (the correctness reference; there is
no reference code to install) on a bounded sample of the same workload: MD
steps of a 20x20x20-cell (32,000-atom) copper box on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2201_01446_gb300 import inputs  # noqa: E402

RC, RCS, SEL = 8.0, 0.5, 256
MD_PER_STEP = 10
DT_FS = 1.0
METRIC = "DP copper atom-steps/s/GPU (fused tabulated vs plain, force err); serve p99 ms"
UNIT = "atom-steps/s"
# nominal FP32 CUDA-core peak of GB300: 152 SMs x 128 FP32 lanes x 2 flop x
# 2.070 GHz; the rooflines use the FMA probe measured in the run itself
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# 16-bit tensor-core products per multiply-add of each fitting mode (FP16 and
# BF16 run at the same kind::f16 rate): FP32 CUDA cores, BF16, three BF16
# pieces (six products), the FP16 pair (h h, h l, l h); mode 4 runs three BF16
# pieces except the dE/dD GEMM (din x w multiply-adds), an FP16 pair
FIT_MODES = ["fp32-cuda-cores", "bf16-tcgen05", "fp32-accurate-tcgen05",
             "near-fp32-tcgen05-fp16-pair", "fp32-accurate-tcgen05-fp16-pair-dE/dD"]


def fit_products(mode, din=2048, w=240):
    """16-bit piece products per multiply-add of the fitting chain, averaged
    over its GEMMs (forward din*w + 2 w*w + w multiply-adds, backward as many,
    the dE/dD GEMM din*w of them)."""
    if mode != 4:
        return {0: 1, 1: 1, 2: 6, 3: 3}[mode]
    tot = 2 * (din * w + 2 * w * w + w)
    return (6 * (tot - din * w) + 3 * din * w) / tot


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=100, help="FCC cells per edge (100 -> 4M atoms)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=5,
                    help="MD steps of the plain untabulated comparator (0: skip)")
    ap.add_argument("--fit-precision", type=int, default=4,
                    choices=[0, 1, 2, 3, 4],
                    help="0 FP32 CUDA cores, 1 BF16 tensor cores, 2 FP32-accurate tensor cores "
                         "(BF16 triples, 6 products), 3 near-FP32 tensor cores (FP16 pairs, "
                         "3 products), 4 BF16 triples with the dE/dD GEMM in FP16 pairs")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving leg (0: skip)")
    ap.add_argument("--serve-capacity-requests", type=int, default=400,
                    help="requests of the closed-loop capacity pass of the serving leg")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--grad-cells", type=int, default=40,
                    help="copper cells per edge of the parameter-gradient leg (0: skip)")
    ap.add_argument("--ref-cells", type=int, default=20,
                    help="FCC cells per edge of the reference arm's oracle sample")
    ap.add_argument("--water-reps", type=int, default=16,
                    help="copies per edge of the 192-atom water box in the water leg (0: skip)")
    ap.add_argument("--water-steps", type=int, default=3,
                    help="timed 10-MD-step blocks of the water leg")
    ap.add_argument("--embed-precision", type=int, default=2,
                    help="tabulated contraction: 0 FP32 CUDA cores, 2 FP32-accurate tensor cores")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id):
        self.proc = None
        self.path = None
        self.dev = dev_id

    def start(self):
        try:
            self.path = tempfile.mktemp(suffix=".csv")
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.dev is not None:
                cmd += ["-i", str(self.dev)]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [q.strip() for q in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_uuid(local):
    try:
        import torch
        p = torch.cuda.get_device_properties(local)
        u = getattr(p, "uuid", None)
        if u is not None:
            s = str(u)
            return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        pass
    return local


# the workload's horizon: one system runs at most 100 MD steps (ten blocks)
# from the initial lattice; the seeded N(0, 0.1) model holds the lattice
# barely at all, so atoms move nearly ballistically at 330 K and, run much
# longer, a few pairs close below the table's r = 0.5 A
MAX_BLOCKS_PER_SYSTEM = 10


def block_segments(nblocks, per_system=MAX_BLOCKS_PER_SYSTEM):
    """Split nblocks bench steps (10-MD-step blocks) into runs of at most
    per_system blocks, one fresh system each."""
    if nblocks < 0 or per_system < 1:
        raise ValueError("bad block count")
    return [min(per_system, nblocks - k) for k in range(0, nblocks, per_system)]


def run_schedule(create, run, destroy, nblocks, keep_last=False,
                 per_system=MAX_BLOCKS_PER_SYSTEM):
    """Run nblocks blocks as block_segments: for each segment create a system
    (initial state), run(system, blocks) and destroy it; with keep_last the
    last segment's system is returned instead of destroyed (None if there was
    no segment)."""
    segs = block_segments(nblocks, per_system)
    last = None
    for k, nb in enumerate(segs):
        s = create()
        run(s, nb)
        if keep_last and k == len(segs) - 1:
            last = s
        else:
            destroy(s)
    return last


def flops_per_unit(M=128, din=2048, w=240):
    """Algorithmic FLOPs (2 per multiply-add) of each phase.
    Per pair within rc: quintic Horner (5 FMA) + 4x1 outer product (4 FMA) per
    embedding column forward; 18 FMA per column backward (value and slope of
    the quintic, dE/dR and dE/ds).  Per atom: the fitting net forward and
    its input gradient, 2 x (din*w + 2*w*w + w) multiply-adds each way."""
    fit = 2 * 2 * (din * w + 2 * w * w + w)
    return {"embed_contract_fwd": ("pair", 2 * 9 * M), "fitting": ("atom", fit),
            "embed_contract_bwd_forces": ("pair", 2 * 18 * M)}


# DRAM bytes per launch of the embedding kernels, from one ncu capture of the
# current build (dram__bytes_read.sum + dram__bytes_write.sum, FCC Cu 256,000
# atoms, scaled per atom: the traffic grows in proportion to the atoms);
# profiles/k_tab_tc_traffic_cu256k.md
TRAFFIC_PER_ATOM = {"embed_contract_fwd": (400750336 + 1346754560) / 256000,
                    "embed_contract_bwd_forces": (1354780672 + 6333184) / 256000}
KERNEL_OF_PHASE = {"embed_contract_fwd": "k_tab_fwd_tc", "embed_contract_bwd_forces": "k_tab_bwd_tc"}


def fp32_peak_probe(stream, local, launches=7, outer=12000):
    """The FP32 FMA probe of the library (every resident thread runs
    independent FMA chains, ~50 ms a launch), timed with CUDA events on the
    stream: median and best TFLOP/s over the launches, and the SM clock
    sampled meanwhile.  This is the FP32 CUDA-core peak the rooflines use."""
    import torch
    from paper_2201_01446_gb300 import dp
    dp.dp_fma_peak_run(outer // 10, C_stream(stream))
    torch.cuda.synchronize()
    ck = Clocks(gpu_uuid(local))
    ck.start()
    res = []
    for _ in range(launches):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fl = dp.dp_fma_peak_run(outer, C_stream(stream))
        e1.record(stream)
        torch.cuda.synchronize()
        res.append(fl / (e0.elapsed_time(e1) / 1e3) / 1e12)
    clk = ck.stop()
    return {"tflops": statistics.median(res), "best_tflops": max(res), "launches": launches,
            "nominal_tflops": FP32_NOMINAL_TFLOPS, "clocks": clk,
            "how": "dp_fma_peak_run: 152 x 8 CTAs of 256 threads, 8 independent FMA chains "
                   "each, CUDA events on the bench stream, median of the launches"}


def plain_roofline(prof, pairs, peak):
    """The plain comparator's embedding kernels against the FP32 CUDA-core
    peak: per pair within rc the net of Eq. 3-5 forward is d1 + d1 d2 + d2 M
    = 10,272 multiply-adds (1-32-64-128), its gradient twice that (the
    backward kernel also recomputes the forward, not counted)."""
    fwd = 2 * 10272
    out = {}
    for k, fl in (("embed_contract_fwd", fwd), ("embed_contract_bwd_forces", 2 * fwd)):
        ms, cnt = prof.get(k, (0.0, 0))
        if cnt:
            a = fl * pairs / (ms / cnt / 1e3) / 1e12
            out[k] = {"achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                      "ms_per_launch": ms / cnt, "flop_per_pair": fl}
    out["bound"] = "alu"
    out["peak_source"] = "FP32 FMA probe measured in this run"
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def cpu_baseline_leg(model_path, xg, t, box, F_gpu, Ei_gpu, n_force=64, n_energy=1024):
    """The FP64 oracle (as it stands) on a bounded sample of the final
    configuration: energies of n_energy atoms and forces on n_force atoms,
    each force needing every centre within rc of the atom.  Returns the
    baseline entry and the sampled errors of the GPU result."""
    import oracle
    m = oracle.Model(model_path)
    tab = oracle.Table(m, 0.01, 2.0)
    ie = inputs.random_subset(len(xg), n_energy, seed=11)
    jf = inputs.random_subset(len(xg), n_force, seed=12)
    t0 = time.perf_counter()
    e_ref, f_ref = oracle.eval_subset(m, tab, RC, RCS, SEL, xg, t, box, ie, jf)
    dt = time.perf_counter() - t0
    # centres evaluated with energy and full backward: each force atom and
    # its neighbors within rc (176 in FCC copper), plus the energy atoms
    centres = n_force * 177 + n_energy
    frmse = float(np.sqrt(((F_gpu[jf] - f_ref) ** 2).mean()))
    frms = float(np.sqrt((f_ref ** 2).mean()))
    emax = float(np.abs(Ei_gpu[ie] - e_ref).max())
    # the stated bars: 1e-6 eV per atom, force RMSE 1e-5 eV/A and at most
    # 1e-3 of the RMS force (the configured model's forces are ~1e-6 eV/A,
    # below the absolute bar, where F = 0 would pass it)
    fbar = min(1e-5, 1e-3 * frms)
    err = {"energy_max_abs_eV_per_atom": emax, "force_rmse_eV_per_A": frmse,
           "force_rms_eV_per_A": frms, "force_bar_eV_per_A": fbar,
           "within_bars": bool(emax < 1e-6 and frmse <= fbar < frms),
           "sample": f"{n_energy} atom energies, forces on {n_force} atoms"}
    base = {"value": centres / dt, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"FP64 oracle on {n_force} force atoms (+{n_energy} energies) of the final "
                      f"{len(xg)}-atom configuration: ~{centres} atom evaluations in {dt:.1f} s"}
    return base, err


def water_leg(args, stream, pg, world, fp32_peak):
    """MD of a two-type water-like box: the seeded 64-molecule box (192 atoms,
    L = 12.417 A) replicated reps^3 times, rc 6 A, sel [46, 92], embedding
    1-25-50-100, fitting 1600-240-240-240-1, dt 0.5 fs, rebuild every 10 steps.
    Atom-steps/s and ns/day with the per-phase times and their fractions of
    the FP32-lane and tensor peaks (the copper figures' definitions)."""
    import torch
    from paper_2201_01446_gb300 import dp
    tmpdir = tempfile.mkdtemp()
    wpath = os.path.join(tmpdir, "water.model")
    inputs.write_seeded_model(wpath, inputs.WATER_SPEC, seed=4, std=0.1)
    r = args.water_reps
    x, t, box = inputs.replicate(*inputs.water_like(64, L=12.417, seed=3), r)
    n = len(x)
    # zero initial velocities: the seeded model holds no molecule together,
    # so thermal motion carries atoms straight into one another (at 330 K a
    # dozen pairs of the 786k atoms came within 0.05 A in 20 fs); the work of
    # a step (lists, pairs, table, fitting) is the same
    v = np.zeros_like(x)
    o = dp.dp_options_default()
    o.fit_precision = args.fit_precision
    o.embed_precision = args.embed_precision
    h = dp.dp_create(wpath, 2, 6.0, 0.5, [46, 92], options=o, stream=C_stream(stream))
    s = dp.dp_system_create(h, x, v, t, [inputs.MASS_O, inputs.MASS_H], box)
    dt = 0.5
    dp.dp_md_step(h, s, MD_PER_STEP, dt)
    torch.cuda.synchronize()
    barrier(pg)
    dp.dp_profile(h, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.water_steps):
        dp.dp_md_step(h, s, MD_PER_STEP, dt)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(pg, e0.elapsed_time(e1))
    prof = dp.dp_profile_read(h)
    stats = dp.dp_stats(h, s)
    dp.dp_system_destroy(s)
    dp.dp_destroy(h)
    steps = MD_PER_STEP * args.water_steps
    value = world * n * steps / (ms / 1e3)
    units = flops_per_unit(M=100, din=1600)
    ach = {k: units[k][1] * (stats["pairs_within_rc"] if units[k][0] == "pair" else n)
           / (prof[k][0] / max(prof[k][1], 1) / 1e3) / 1e12 for k in units if prof[k][1]}
    nprod = fit_products(args.fit_precision, din=1600)
    bf16 = measured_peaks().get("bf16_tflops_sustained") or 1700.0
    return {"value": value, "unit": UNIT, "natoms": n, "md_steps": steps, "dt_fs": dt,
            "ns_per_day": value / world / n * dt * 86400 * 1e-6,
            "ms_per_md_step": ms / steps,
            "phases_ms_per_launch": {k: v[0] / max(v[1], 1) for k, v in prof.items()},
            "phases_achieved_tflops": ach,
            "embed_fwd_frac_of_fp32_peak": ach.get("embed_contract_fwd", 0.0) / fp32_peak,
            "fitting_frac_of_tensor_peak": ach.get("fitting", 0.0) / (bf16 / nprod),
            "pairs_within_rc": stats["pairs_within_rc"],
            "workload": f"water-like 64-molecule box replicated {r}^3 ({n} atoms), rc 6 A, "
                        "sel [46, 92], 1-25-50-100 / 1600-240-240-240-1, tabulated h=0.01 s<=2, "
                        "zero initial velocities, dt 0.5 fs, rebuild every 10, skin 2 A"}


def serve_leg(args, cu_model, pg):
    """The serving loop (request stream with admission, several slots): the
    seeded mix of copper (500-500,000 atoms, log-uniform) and water-like
    (192-24,576 atoms) boxes, half energy/force evaluations and half 50-step
    MD runs, under the 150 GB device budget.  A closed-loop pass over the
    first requests of the stream measures capacity; the open-loop pass then
    offers the whole Poisson stream at 70% of it and reports latency from
    arrival, and the most device memory the library held meanwhile."""
    from paper_2201_01446_gb300 import dp, serve
    wpath = os.path.join(os.path.dirname(cu_model), "water.model")
    inputs.write_seeded_model(wpath, inputs.WATER_SPEC, seed=4, std=0.1)

    def opts(s_max):
        o = dp.dp_options_default()
        o.fit_precision = args.fit_precision
        o.embed_precision = args.embed_precision
        o.s_max = s_max
        return o

    # table domain s <= 2.0 (r >= 0.5 A) for both models
    models = {"cu": serve.ModelCfg(cu_model, 1, RC, RCS, [SEL], opts(2.0)),
              "water": serve.ModelCfg(wpath, 2, 6.0, 0.5, [46, 92], opts(2.0), {"M": 100})}
    specs = inputs.serve_requests(args.serve_requests, seed=5)
    budget = 150e9
    srv = serve.Server(models, slots=args.serve_slots, budget_bytes=budget)
    ncap = min(len(specs), args.serve_capacity_requests)
    closed = srv.run(serve.make_requests(specs[:ncap]), np.zeros(ncap))
    capacity = ncap / closed["makespan_s"]
    lam = 0.7 * capacity
    base = dp.dp_memory(reset_peak=True)["process"]
    st = srv.run(serve.make_requests(specs), inputs.poisson_arrivals(len(specs), lam, seed=6))
    mem = dp.dp_memory()
    return {"p50_ms": st["p50_ms"], "p99_ms": max_over_ranks(pg, st["p99_ms"]), "unit": "ms",
            "requests": len(specs), "errors": st["errors"] + closed["errors"],
            "arrival_rate_per_s": lam, "capacity_req_per_s": capacity,
            "capacity_sample": f"closed loop over the first {ncap} requests",
            "atom_steps_per_s": st["atom_steps_per_s"], "slots": args.serve_slots,
            "makespan_s": st["makespan_s"],
            "packed_calls": st["packed_calls"], "packed_requests": st["packed_requests"],
            "budget_bytes": budget, "admission_peak_bytes": st["peak_budget_bytes"],
            "device_peak_bytes": mem["peak"] - base, "trims": st["trims"],
            "mix": "Cu 500-500k atoms log-uniform + water 192*2^k (k<8), half eval half MD "
                   "(50 steps; water MD from rest), Poisson arrivals at 0.7 x closed-loop "
                   "capacity; queued requests of one model and kind (MD: same steps) packed up "
                   "to 32768 atoms per call"}


def grad_leg(args, model_path, stream):
    """Parameter gradients (dE/d fitting parameters and table coefficients)
    of one copper box through dp_param_grad: wall time of the synchronous
    call (host coordinates in, gradients out) after one warm-up call."""
    from paper_2201_01446_gb300 import dp
    o = dp.dp_options_default()
    o.embed_precision = args.embed_precision
    o.fit_precision = args.fit_precision
    h = dp.dp_create(model_path, 1, RC, RCS, [SEL], options=o, stream=C_stream(stream))
    try:
        x, t, box = inputs.fcc_copper(args.grad_cells, sigma=0.05, seed=7)
        dp.dp_param_grad(h, x, t, box, table=args.embed_precision == 2)
        reps = 3
        t0 = time.perf_counter()
        for _ in range(reps):
            dp.dp_param_grad(h, x, t, box, table=args.embed_precision == 2)
        ms = (time.perf_counter() - t0) / reps * 1e3
        nf, nt = dp.dp_param_sizes(h)
    finally:
        dp.dp_destroy(h)
    return {"natoms": len(x), "ms_per_call": ms, "atoms_per_s": len(x) / (ms / 1e3),
            "n_fit_params": nf, "n_table_params": nt if args.embed_precision == 2 else 0,
            "timing": "host wall clock of the synchronous call, coordinates in, gradients out"}


def run_reference(args, world, rank, pg):
    if rank != 0:
        return 0
    import oracle
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "cu.model")
        inputs.write_seeded_model(path, inputs.COPPER_SPEC, seed=0, std=0.1)
        m = oracle.Model(path)
        tab = oracle.Table(m, 0.01, 2.0)
        x, t, box = inputs.fcc_copper(args.ref_cells, sigma=0.0)
        v = inputs.maxwell_velocities(np.full(len(x), inputs.MASS_CU), 330.0, seed=2)
        masses = [inputs.MASS_CU]
        x, v, f, _ = oracle.md(m, tab, RC, RCS, SEL, x, v, t, masses, box, DT_FS, 0)
        for _ in range(args.warmup):
            x, v, f, _ = oracle.md(m, tab, RC, RCS, SEL, x, v, t, masses, box, DT_FS, 1, f=f)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            x, v, f, _ = oracle.md(m, tab, RC, RCS, SEL, x, v, t, masses, box, DT_FS, 1, f=f)
        dt = time.perf_counter() - t0
    value = len(x) * args.steps / dt
    cores = oracle.get_threads()
    sample = (f"FP64 oracle velocity-Verlet, {len(x)}-atom copper box ({args.ref_cells}^3 cells), "
              "1 MD step per bench step")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"FCC Cu 330 K, rc 8 A, seeded N(0,0.1) DP-SE_a model, "
                                   f"sample of {len(x)} atoms", "md_steps_per_step": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank, pg)
    import torch
    from paper_2201_01446_gb300 import dp
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    tmpdir = tempfile.mkdtemp()
    model = os.path.join(tmpdir, "cu.model")
    inputs.write_seeded_model(model, inputs.COPPER_SPEC, seed=0, std=0.1)
    x, t, box = inputs.fcc_copper(args.cells, sigma=0.0)
    n = len(x)
    v = inputs.maxwell_velocities(np.full(n, inputs.MASS_CU), 330.0, seed=2 + rank)
    masses = [inputs.MASS_CU]
    opt = dp.dp_options_default()
    opt.fit_precision = args.fit_precision
    opt.embed_precision = args.embed_precision
    h = dp.dp_create(model, 1, RC, RCS, [SEL], options=opt, stream=C_stream(stream))
    # warm-up on a system of its own, then the timed blocks; no system runs
    # past the workload's 100 MD steps (block_segments), each new one starts
    # from the initial lattice and velocities and is created outside the
    # CUDA-event windows
    run_schedule(lambda: dp.dp_system_create(h, x, v, t, masses, box),
                 lambda s, nb: dp.dp_md_step(h, s, MD_PER_STEP * nb, DT_FS),
                 dp.dp_system_destroy, args.warmup)
    fp32 = fp32_peak_probe(stream, local)
    torch.cuda.synchronize()
    barrier(pg)
    torch.cuda.synchronize()
    clocks = Clocks(gpu_uuid(local))
    clocks.start()
    acc = {"ms": 0.0, "launches": 0, "prof": {k: [0.0, 0] for k in dp.PHASES}}

    def timed_segment(s, nb):
        # one CUDA-event window per segment on the library's stream; the
        # system's creation (list build and first force evaluation) is outside
        torch.cuda.synchronize()
        barrier(pg)
        torch.cuda.synchronize()
        l0 = dp.dp_stats(h, s)["kernel_launches"]
        dp.dp_profile(h, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dp.dp_md_step(h, s, MD_PER_STEP * nb, DT_FS)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(pg)
        torch.cuda.synchronize()
        acc["ms"] += e0.elapsed_time(e1)
        acc["launches"] += dp.dp_stats(h, s)["kernel_launches"] - l0
        for k, (pm, pl) in dp.dp_profile_read(h).items():
            acc["prof"][k][0] += pm
            acc["prof"][k][1] += pl
        dp.dp_profile(h, False)

    s = run_schedule(lambda: dp.dp_system_create(h, x, v, t, masses, box), timed_segment,
                     dp.dp_system_destroy, args.steps, keep_last=True)
    ck = clocks.stop()
    prof = {k: tuple(vv) for k, vv in acc["prof"].items()}
    ms = acc["ms"]
    ms_max = max_over_ranks(pg, ms)
    stats = dp.dp_stats(h, s)
    launches = acc["launches"]
    value = world * n * MD_PER_STEP * args.steps / (ms_max / 1e3)
    # roofline of the dominant kernel: the phases of one launch each (the
    # embedding forward and backward) are single kernels; the fitting phase is
    # a chain of seven GEMM launches per row chunk and is reported beside it
    units = flops_per_unit()
    peaks = measured_peaks()
    per_launch = {k: prof[k][0] / max(prof[k][1], 1) for k in prof}

    def phase_achieved(k):
        kind, fl = units[k]
        return fl * (stats["pairs_within_rc"] if kind == "pair" else n) / (per_launch[k] / 1e3) / 1e12

    single = [k for k in KERNEL_OF_PHASE if prof.get(k, (0, 0))[1]]
    dom = max(single, key=lambda k: per_launch[k])
    achieved = phase_achieved(dom)
    traffic = TRAFFIC_PER_ATOM[dom] * n if args.embed_precision == 2 else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32["tflops"],
                "unit": "TFLOP/s", "frac": achieved / fp32["tflops"], "traffic": traffic,
                "kernel": KERNEL_OF_PHASE[dom] if args.embed_precision == 2 else dom,
                "peak_source": "FP32 FMA probe measured in this run (fp32_peak); nominal "
                               "152 SMs x 128 lanes x 2 x 2.070 GHz = %.1f" % FP32_NOMINAL_TFLOPS,
                "note": "achieved counts the method's per-pair FLOPs (2304 per pair within rc); "
                        "the interval contraction inside runs on tcgen05"}
    if args.fit_precision > 0 and prof.get("fitting", (0, 0))[1]:
        # the fitting chain against the peak of the arithmetic it computes in:
        # BF16 products for the BF16 mode; for the split modes, whose every
        # multiply-add is six BF16 (three FP16) piece products, the 16-bit
        # peak / 6 (/ 3)
        nprod = fit_products(args.fit_precision)
        bf16 = peaks.get("bf16_tflops_sustained") or 1700.0
        fa = phase_achieved("fitting")
        roofline["fitting_chain"] = {
            "bound": "tensor", "achieved": fa, "peak": bf16 / nprod, "unit": "TFLOP/s",
            "frac": fa / (bf16 / nprod), "executed_16bit_tflops": fa * nprod, "bf16_peak": bf16,
            "ms_per_launch": per_launch["fitting"],
            "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
                            + (" / %.3g piece products" % nprod if nprod > 1 else "")
                            if peaks else "fallback 1.7 PFLOP/s sustained")}
    roofline["phases_ms_per_launch"] = {k: prof[k][0] / max(prof[k][1], 1) for k in prof}
    roofline["phases_achieved_tflops"] = {
        k: units[k][1] * (stats["pairs_within_rc"] if units[k][0] == "pair" else n)
        / (prof[k][0] / max(prof[k][1], 1) / 1e3) / 1e12 for k in units if prof[k][1]}
    xg, vg, fg = dp.dp_system_get(h, s, n)
    dp.dp_system_destroy(s)
    # the plain untabulated FP32 comparator on the same final configuration
    plain = None
    if args.plain_steps > 0:
        popt = dp.dp_options_default()
        popt.tabulated = 0
        popt.fit_precision = args.fit_precision
        hp = dp.dp_create(model, 1, RC, RCS, [SEL], options=popt, stream=C_stream(stream))
        # from the initial lattice and velocities, as every timed system
        sp = dp.dp_system_create(hp, x, v, t, masses, box)
        dp.dp_md_step(hp, sp, 1, DT_FS)
        torch.cuda.synchronize()
        barrier(pg)
        dp.dp_profile(hp, True)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        dp.dp_md_step(hp, sp, args.plain_steps, DT_FS)
        p1.record(stream)
        torch.cuda.synchronize()
        pms = max_over_ranks(pg, p0.elapsed_time(p1))
        pprof = dp.dp_profile_read(hp)
        ppairs = dp.dp_stats(hp, sp)["pairs_within_rc"]
        dp.dp_system_destroy(sp)
        dp.dp_destroy(hp)
        plain = {"value": world * n * args.plain_steps / (pms / 1e3), "unit": UNIT,
                 "md_steps": args.plain_steps, "ms_per_md_step": pms / args.plain_steps,
                 "phases_ms_per_launch": {k: v[0] / max(v[1], 1) for k, v in pprof.items()},
                 "speedup_of_tabulated": (value / world) / (n * args.plain_steps / (pms / 1e3)),
                 "roofline": plain_roofline(pprof, ppairs, fp32["tflops"]),
                 "start": "initial lattice and velocities (as each timed tabulated system), after one untimed MD step"}
    # e2e: host buffers in, 10 MD steps, host buffers out (pinned host
    # memory, allocated and filled before the timed region)
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        xh = torch.from_numpy(np.ascontiguousarray(x, np.float64)).pin_memory()
        vh = torch.from_numpy(np.ascontiguousarray(v, np.float64)).pin_memory()
        outs = tuple(torch.empty((n, 3), dtype=torch.float64).pin_memory() for _ in range(3))
        barrier(pg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            se = dp.dp_system_create(h, xh, vh, t, masses, box)
            dp.dp_md_step(h, se, MD_PER_STEP, DT_FS)
            dp.dp_system_get(h, se, n, out=outs)
            dp.dp_system_destroy(se)
        torch.cuda.synchronize()
        te = max_over_ranks(pg, time.perf_counter() - t0)
        e2e = {"value": world * n * MD_PER_STEP * args.e2e_steps / te, "unit": UNIT,
               "h2d_bytes_per_step": int(n * (3 * 8 + 3 * 8 + 4) + 9 * 8 + 8),
               "d2h_bytes_per_step": int(n * 3 * 8 * 3)}
    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu:
        E, F, V, Ei = dp.dp_compute(h, xg, t, box, atom_energy=True)
        cpu, accuracy = cpu_baseline_leg(model, xg, t, box, F, Ei)
    dp.dp_destroy(h)
    grad_info = grad_leg(args, model, stream) if args.grad_cells > 0 else None
    water_info = None
    if args.water_reps > 0:
        try:
            water_info = water_leg(args, stream, pg, world, fp32["tflops"])
        except dp.DPError as e:  # a library error of this leg is reported, not fatal
            water_info = {"error": str(e)}
    serve_info = serve_leg(args, model, pg) if args.serve_requests > 0 else None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded model and lattice)",
                "config": {"workload": f"FCC Cu {args.cells}^3 cells ({n} atoms) 330 K, DP-SE_a "
                                       "1-32-64-128 / 2048-240-240-240-1, rc 8 A, tabulated "
                                       "h=0.01 s<=2, velocity-Verlet dt 1 fs, rebuild every 10, skin 2 A",
                           "md_steps_per_step": MD_PER_STEP, "natoms": n,
                           "fit_precision": FIT_MODES[args.fit_precision], "l2": "inputs larger than L2",
                           "ns_per_day": value / world / n * DT_FS * 86400 * 1e-6,
                           "parallelism": f"replicas x{world}",
                           "systems": len(block_segments(args.steps)),
                           "timing": "CUDA events around the MD blocks of each system (at most "
                                     f"{MAX_BLOCKS_PER_SYSTEM * MD_PER_STEP} MD steps from the "
                                     "initial state), summed; system creation (list build and "
                                     "first force evaluation) excluded from value, included in "
                                     "e2e"},
                "gpu_launches": launches, "roofline": roofline, "fp32_peak": fp32, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": ck, "accuracy_vs_oracle": accuracy, "plain": plain,
                "serve": serve_info, "param_grad": grad_info, "water": water_info,
                "stats": stats}
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def C_stream(stream):
    import ctypes
    return ctypes.c_void_p(stream.cuda_stream)


if __name__ == "__main__":
    sys.exit(main())
