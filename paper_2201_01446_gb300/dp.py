"""Thin ctypes binding of libdp.so (include/dp.h).

The functions below carry the C names and only marshal arguments: every step
of the computation runs in the library's CUDA kernels.  Arrays may be numpy
arrays (host memory) or CUDA torch tensors (device memory, the call then runs
on the handle's stream, by default torch's current stream).  There is no CPU
fallback: if the library cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

STATUS = {0: "DP_OK", 1: "DP_ERR_ARG", 2: "DP_ERR_MODEL", 3: "DP_ERR_CUDA", 4: "DP_ERR_OOM",
          5: "DP_ERR_SEL_OVERFLOW", 6: "DP_ERR_TABLE_RANGE", 7: "DP_ERR_BOX",
          8: "DP_ERR_TIMEOUT", 9: "DP_ERR_UNIMPLEMENTED", 10: "DP_ERR_SKIN",
          11: "DP_ERR_NONFINITE", 12: "DP_ERR_CAPACITY"}


class DPError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class dp_options(C.Structure):
    _fields_ = [("tabulated", C.c_int), ("fit_precision", C.c_int), ("table_step", C.c_double),
                ("s_max", C.c_double), ("skin", C.c_double), ("rebuild_every", C.c_int),
                ("embed_precision", C.c_int), ("tanh_table", C.c_int), ("md_graphs", C.c_int),
                ("s_ext", C.c_double), ("ext_stride", C.c_int)]


class dp_thermo(C.Structure):
    _fields_ = [("step", C.c_int64), ("kinetic", C.c_double), ("potential", C.c_double),
                ("temperature", C.c_double), ("pressure", C.c_double),
                ("virial", C.c_double * 9)]


EXPORTS = ["dp_options_default", "dp_create", "dp_destroy", "dp_last_error", "dp_set_stream",
           "dp_compute", "dp_system_create", "dp_system_destroy", "dp_system_get",
           "dp_system_step", "dp_md_step", "dp_state_save", "dp_state_load",
           "dp_neighbor_pairs", "dp_table_coeffs", "dp_descriptor", "dp_version",
           "dp_profile", "dp_profile_read", "dp_stats", "dp_neighbor_pairs_static", "dp_fitting",
           "dp_param_sizes", "dp_param_grad", "dp_get_params", "dp_set_params", "dp_compute_batch",
           "dp_system_create_batch", "dp_system_batch_size", "dp_fma_peak_run",
           "dp_memory", "dp_trim"]

DP_NPHASE = 5
PHASES = ["neighbor_build", "embed_contract_fwd", "fitting", "embed_contract_bwd_forces",
          "integrate_reduce"]


def _load():
    if os.environ.get("DP_SKIP_BUILD") != "1":
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libdp.so not found at {_build.LIB}; build it with build.build()")
    L = C.CDLL(_build.LIB)
    vp, i32p, i64p, dp_ = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.c_void_p
    d, i, i64 = C.c_double, C.c_int, C.c_int64
    sig = {
        "dp_options_default": (None, [C.POINTER(dp_options)]),
        "dp_create": (i, [C.c_char_p, i, vp, d, d, vp, C.POINTER(dp_options), vp,
                          C.POINTER(vp)]),
        "dp_destroy": (None, [vp]),
        "dp_last_error": (C.c_char_p, [vp]),
        "dp_set_stream": (i, [vp, vp]),
        "dp_compute": (i, [vp, i64, dp_, dp_, dp_, i, dp_, dp_, dp_, dp_]),
        "dp_system_create": (i, [vp, i64, dp_, dp_, dp_, dp_, dp_, i, C.POINTER(vp)]),
        "dp_system_destroy": (None, [vp]),
        "dp_system_get": (i, [vp, dp_, dp_, dp_, i]),
        "dp_system_step": (i64, [vp]),
        "dp_md_step": (i, [vp, vp, i, d, C.POINTER(dp_thermo)]),
        "dp_state_save": (i, [vp, C.c_char_p]),
        "dp_state_load": (i, [vp, C.c_char_p, C.POINTER(vp)]),
        "dp_neighbor_pairs": (i, [vp, i64, dp_, dp_, d, i64, i32p, i64p]),
        "dp_table_coeffs": (i, [vp, i, i, vp, i32p]),
        "dp_descriptor": (i, [vp, i64, dp_, dp_, dp_, vp]),
        "dp_version": (C.c_char_p, []),
        "dp_profile": (i, [vp, i]),
        "dp_profile_read": (i, [vp, vp, vp]),
        "dp_stats": (i, [vp, vp, vp]),
        "dp_neighbor_pairs_static": (i, [i64, vp, vp, d, i64, vp, i64p, vp]),
        "dp_fitting": (i, [vp, i64, vp, vp, vp, vp]),
        "dp_param_sizes": (i, [vp, i64p, i64p]),
        "dp_param_grad": (i, [vp, i64, dp_, dp_, dp_, vp, vp, vp]),
        "dp_get_params": (i, [vp, vp, vp]),
        "dp_compute_batch": (i, [vp, i, vp, vp, vp, vp, vp, vp, vp]),
        "dp_system_create_batch": (i, [vp, i, vp, vp, vp, vp, vp, vp, C.POINTER(vp)]),
        "dp_set_params": (i, [vp, vp, vp]),
        "dp_system_batch_size": (i, [vp]),
        "dp_fma_peak_run": (i, [i64, vp, C.POINTER(d)]),
        "dp_memory": (i, [vp, i64p, i64p, i64p, i]),
        "dp_trim": (i, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


lib = _load()


# ---------------------------------------------------------------- marshalling
def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, keepalive, is_device) of a numpy array or torch tensor."""
    if a is None:
        return None, None, False
    if _is_torch(a):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.float32: torch.float32}[dtype]
        assert a.dtype == tdt and a.is_contiguous(), "tensor must be contiguous of the right dtype"
        return C.c_void_p(a.data_ptr()), a, a.is_cuda
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(C.c_void_p), arr, False


def _check(code, h=None):
    if code != 0:
        raise DPError(code, lib.dp_last_error(h).decode(errors="replace"))


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def dp_options_default():
    o = dp_options()
    lib.dp_options_default(C.byref(o))
    return o


def dp_version() -> str:
    return lib.dp_version().decode()


def dp_create(model_path, ntypes, rc, rcs, sel, type_map=None, options=None, stream="torch"):
    sel = np.ascontiguousarray(np.atleast_1d(sel), np.int32)
    tm = None if type_map is None else np.ascontiguousarray(type_map, np.int32)
    opt = options if options is not None else dp_options_default()
    st = _torch_stream() if stream == "torch" else stream
    out = C.c_void_p()
    code = lib.dp_create(str(model_path).encode(), int(ntypes),
                         tm.ctypes.data_as(C.c_void_p) if tm is not None else None, float(rc),
                         float(rcs), sel.ctypes.data_as(C.c_void_p), C.byref(opt), st,
                         C.byref(out))
    _check(code, None)
    return out


def dp_destroy(h):
    lib.dp_destroy(h)


def dp_set_stream(h, stream):
    _check(lib.dp_set_stream(h, stream), h)


def dp_compute(h, coords, types, box, atom_energy=False):
    """Energy (float), forces [N,3], virial [3,3], optional per-atom energy.

    numpy inputs: host call, numpy outputs.  CUDA tensors: device call,
    torch outputs on the same device (energy/virial as tensors)."""
    dev = _is_torch(coords) and coords.is_cuda
    n = int(coords.shape[0])
    if dev:
        import torch
        energy = torch.zeros(1, dtype=torch.float64, device=coords.device)
        forces = torch.empty((n, 3), dtype=torch.float64, device=coords.device)
        virial = torch.empty(9, dtype=torch.float64, device=coords.device)
        ae = torch.empty(n, dtype=torch.float64, device=coords.device) if atom_energy else None
        box_t = box if _is_torch(box) else torch.as_tensor(np.asarray(box, np.float64),
                                                           device=coords.device)
        args = [_ptr(coords, np.float64), _ptr(types, np.int32), _ptr(box_t, np.float64)]
        outs = [C.c_void_p(energy.data_ptr()), C.c_void_p(forces.data_ptr()),
                C.c_void_p(virial.data_ptr()), C.c_void_p(ae.data_ptr()) if ae is not None else None]
        _check(lib.dp_compute(h, n, args[0][0], args[1][0], args[2][0], 1, *outs), h)
        return energy, forces, virial.view(3, 3), ae
    energy = np.zeros(1)
    forces = np.zeros((max(n, 1), 3))
    virial = np.zeros(9)
    ae = np.zeros(max(n, 1)) if atom_energy else None
    c, ck, _ = _ptr(coords, np.float64)
    t, tk, _ = _ptr(types, np.int32)
    b, bk, _ = _ptr(box, np.float64)
    _check(lib.dp_compute(h, n, c, t, b, 0, energy.ctypes.data_as(C.c_void_p),
                          forces.ctypes.data_as(C.c_void_p), virial.ctypes.data_as(C.c_void_p),
                          ae.ctypes.data_as(C.c_void_p) if ae is not None else None), h)
    return float(energy[0]), forces[:n], virial.reshape(3, 3), (ae[:n] if ae is not None else None)


def dp_system_create(h, x, v, types, masses, box):
    dev = _is_torch(x) and x.is_cuda
    n = int(x.shape[0])
    out = C.c_void_p()
    if dev:
        import torch
        m = masses if _is_torch(masses) else torch.as_tensor(np.asarray(masses, np.float64),
                                                             device=x.device)
        b = box if _is_torch(box) else torch.as_tensor(np.asarray(box, np.float64),
                                                       device=x.device)
        ptrs = [_ptr(a, dt) for a, dt in ((x, np.float64), (v, np.float64), (types, np.int32),
                                           (m, np.float64), (b, np.float64))]
        _check(lib.dp_system_create(h, n, *[p[0] for p in ptrs], 1, C.byref(out)), h)
    else:
        ptrs = [_ptr(a, dt) for a, dt in ((x, np.float64), (v, np.float64), (types, np.int32),
                                           (masses, np.float64), (box, np.float64))]
        _check(lib.dp_system_create(h, n, *[p[0] for p in ptrs], 0, C.byref(out)), h)
    return out


def dp_system_create_batch(h, systems, masses):
    """Several systems [(x [n, 3], v [n, 3], types [n], box [3, 3]), ...] as
    one MD system (host arrays); dp_system_get returns them concatenated."""
    nsys = len(systems)
    counts = np.array([len(np.reshape(x, (-1, 3))) for x, _, _, _ in systems], np.int64)
    cat = lambda k, shape, dt: np.ascontiguousarray(  # noqa: E731
        np.concatenate([np.reshape(sy[k], shape) for sy in systems]) if nsys else np.zeros(0), dt)
    x, v = cat(0, (-1, 3), np.float64), cat(1, (-1, 3), np.float64)
    t = cat(2, (-1,), np.int32)
    boxes = np.ascontiguousarray(np.stack([np.asarray(sy[3], np.float64).reshape(3, 3)
                                           for sy in systems]) if nsys else np.zeros((1, 3, 3)))
    m = np.ascontiguousarray(masses, np.float64)
    out = C.c_void_p()
    _check(lib.dp_system_create_batch(h, nsys, counts.ctypes.data_as(C.c_void_p),
                                      x.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p),
                                      t.ctypes.data_as(C.c_void_p), m.ctypes.data_as(C.c_void_p),
                                      boxes.ctypes.data_as(C.c_void_p), C.byref(out)), h)
    return out


def dp_system_destroy(s):
    lib.dp_system_destroy(s)


def dp_system_step(s) -> int:
    return int(lib.dp_system_step(s))


def dp_system_get(h, s, n, x=True, v=True, f=True, out=None):
    """Host copies (numpy) of x, v, f; or, with out=(x, v, f) of CUDA tensors,
    device-to-device copies into them; or, with out of host arrays (numpy or
    CPU tensors, e.g. pinned), host copies into them."""
    if out is not None:
        dev = any(_is_torch(t) and t.is_cuda for t in out if t is not None)
        ptrs = [(C.c_void_p(t.data_ptr()) if _is_torch(t) else t.ctypes.data_as(C.c_void_p))
                if t is not None else None for t in out]
        _check(lib.dp_system_get(s, *ptrs, 1 if dev else 0), h)
        return out
    arrs = [np.zeros((max(n, 1), 3)) if want else None for want in (x, v, f)]
    _check(lib.dp_system_get(s, *[a.ctypes.data_as(C.c_void_p) if a is not None else None
                                  for a in arrs], 0), h)
    return tuple(a[:n] if a is not None else None for a in arrs)


def dp_md_step(h, s, nsteps, dt_fs, thermo=False):
    """nsteps velocity-Verlet steps; with thermo, the records (step, KE, PE,
    T, P) as [nsteps, 5], or [nsteps, nsys, 5] for a batch system."""
    nsys = int(lib.dp_system_batch_size(s))
    th = (dp_thermo * (max(nsteps, 1) * max(nsys, 1)))() if thermo else None
    _check(lib.dp_md_step(h, s, int(nsteps), float(dt_fs), th), h)
    if not thermo:
        return None
    rec = np.array([(t.step, t.kinetic, t.potential, t.temperature, t.pressure)
                    for t in th[:nsteps * max(nsys, 1)]]).reshape(-1, 5)
    return rec.reshape(nsteps, nsys, 5) if nsys else rec


def dp_state_save(h, s, path):
    _check(lib.dp_state_save(s, str(path).encode()), h)


def dp_state_load(h, path):
    out = C.c_void_p()
    _check(lib.dp_state_load(h, str(path).encode(), C.byref(out)), h)
    return out


def dp_neighbor_pairs(h, coords, box, rlist):
    c, ck, _ = _ptr(coords, np.float64)
    b, bk, _ = _ptr(box, np.float64)
    n = int(np.asarray(coords).shape[0])
    cnt = C.c_int64()
    _check(lib.dp_neighbor_pairs(h, n, c, b, float(rlist), 0, None, C.byref(cnt)), h)
    out = np.zeros((max(cnt.value, 1), 5), np.int32)
    _check(lib.dp_neighbor_pairs(h, n, c, b, float(rlist), cnt.value,
                                 out.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(cnt)), h)
    return out[:cnt.value]


def dp_table_coeffs(h, ti=0, tj=0, M=None):
    n = C.c_int32()
    _check(lib.dp_table_coeffs(h, ti, tj, None, C.byref(n)), h)
    if M is None:
        raise ValueError("M (embedding width) is required")
    out = np.zeros((n.value, 6, M), np.float32)
    _check(lib.dp_table_coeffs(h, ti, tj, out.ctypes.data_as(C.c_void_p), C.byref(n)), h)
    return out


def dp_descriptor(h, coords, types, box, M):
    n = int(np.asarray(coords).shape[0])
    T = np.zeros((max(n, 1), 4, M), np.float32)
    c, ck, _ = _ptr(coords, np.float64)
    t, tk, _ = _ptr(types, np.int32)
    b, bk, _ = _ptr(box, np.float64)
    _check(lib.dp_descriptor(h, n, c, t, b, T.ctypes.data_as(C.c_void_p)), h)
    return T[:n]


def dp_profile(h, enable=True):
    _check(lib.dp_profile(h, 1 if enable else 0), h)


def dp_profile_read(h):
    """{phase: (ms, launches)} of the phases timed since dp_profile(h, True)."""
    ms = np.zeros(DP_NPHASE)
    cnt = np.zeros(DP_NPHASE, np.int64)
    _check(lib.dp_profile_read(h, ms.ctypes.data_as(C.c_void_p), cnt.ctypes.data_as(C.c_void_p)), h)
    return {PHASES[k]: (float(ms[k]), int(cnt[k])) for k in range(DP_NPHASE)}


def dp_stats(h, s=None):
    out = np.zeros(6, np.int64)
    _check(lib.dp_stats(h, s, out.ctypes.data_as(C.c_void_p)), h)
    return dict(natoms=int(out[0]), list_capacity=int(out[1]), max_list=int(out[2]),
                pairs_within_rc=int(out[3]), cells=int(out[4]), kernel_launches=int(out[5]))


def dp_neighbor_pairs_static(coords, box, rlist, stream=None, out=None):
    """Pair rows (i, j, n0, n1, n2) of a CUDA float64 tensor of positions,
    computed by the library without allocating device memory (its scratch
    is a fixed array).  Without out, the output tensor is allocated here by
    torch, on the caller's side of the call (a first call returns only the
    count) and the rows are returned.  With out (a CUDA int32 tensor [cap][5],
    cap >= 0), one call writes at most cap rows into it and (out, total
    count) is returned."""
    import torch
    assert coords.is_cuda and coords.dtype == torch.float64 and coords.is_contiguous()
    n = int(coords.shape[0])
    b = np.ascontiguousarray(box, np.float64)
    cnt = C.c_int64()
    if out is not None:
        assert out.is_cuda and out.dtype == torch.int32 and out.is_contiguous()
        cap = int(out.shape[0])
        _check(lib.dp_neighbor_pairs_static(n, C.c_void_p(coords.data_ptr()),
                                            b.ctypes.data_as(C.c_void_p), float(rlist), cap,
                                            C.c_void_p(out.data_ptr()) if cap else None,
                                            C.byref(cnt), stream), None)
        return out, cnt.value
    _check(lib.dp_neighbor_pairs_static(n, C.c_void_p(coords.data_ptr()),
                                        b.ctypes.data_as(C.c_void_p), float(rlist), 0, None,
                                        C.byref(cnt), stream), None)
    out = torch.empty((max(cnt.value, 1), 5), dtype=torch.int32, device=coords.device)
    _check(lib.dp_neighbor_pairs_static(n, C.c_void_p(coords.data_ptr()),
                                        b.ctypes.data_as(C.c_void_p), float(rlist), cnt.value,
                                        C.c_void_p(out.data_ptr()), C.byref(cnt), stream), None)
    return out[:cnt.value]


def dp_memory(h=None, reset_peak=False):
    """{"handle": bytes of h (None without h), "process": bytes held by the
    library, "peak": most held since the last reset} (host counters)."""
    hb, pb, pk = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib.dp_memory(h, C.byref(hb) if h is not None else None, C.byref(pb), C.byref(pk),
                         1 if reset_peak else 0), h)
    return {"handle": hb.value if h is not None else None, "process": pb.value, "peak": pk.value}


def dp_trim(h):
    """Free the handle's caches (work area, kept system buffers, scratch)."""
    _check(lib.dp_trim(h), h)


def dp_fma_peak_run(outer, stream=None):
    """Launch the FP32 FMA probe once on the stream (default: torch's
    current one); returns the FLOPs of the launch."""
    fl = C.c_double()
    _check(lib.dp_fma_peak_run(int(outer), stream if stream is not None else _torch_stream(),
                               C.byref(fl)), None)
    return fl.value


def dp_compute_batch(h, systems):
    """Several systems [(coords [n, 3], types [n], box [3, 3]), ...] in one
    evaluation (host arrays): (energies [nsys], [forces [n, 3] per system],
    virials [nsys, 3, 3])."""
    nsys = len(systems)
    counts = np.array([len(np.atleast_2d(x)) if np.size(x) else 0 for x, _, _ in systems], np.int64)
    n = int(counts.sum())
    x = np.ascontiguousarray(np.concatenate([np.reshape(x, (-1, 3)) for x, _, _ in systems])
                             if nsys else np.zeros((0, 3)), np.float64)
    t = np.ascontiguousarray(np.concatenate([np.ravel(t) for _, t, _ in systems])
                             if nsys else np.zeros(0), np.int32)
    boxes = np.ascontiguousarray(np.stack([np.asarray(b, np.float64).reshape(3, 3)
                                           for _, _, b in systems]) if nsys else np.zeros((1, 3, 3)))
    e = np.zeros(max(nsys, 1))
    f = np.zeros((max(n, 1), 3))
    v = np.zeros((max(nsys, 1), 9))
    _check(lib.dp_compute_batch(h, nsys, counts.ctypes.data_as(C.c_void_p),
                                x.ctypes.data_as(C.c_void_p), t.ctypes.data_as(C.c_void_p),
                                boxes.ctypes.data_as(C.c_void_p), e.ctypes.data_as(C.c_void_p),
                                f.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p)), h)
    off = np.concatenate([[0], np.cumsum(counts)])
    return e[:nsys], [f[off[q]:off[q + 1]] for q in range(nsys)], v[:nsys].reshape(nsys, 3, 3)


def dp_param_sizes(h):
    """(n_fit, n_table): doubles of the two parameter-gradient arrays."""
    nf, nt = C.c_int64(), C.c_int64()
    _check(lib.dp_param_sizes(h, C.byref(nf), C.byref(nt)), h)
    return nf.value, nt.value


def dp_param_grad(h, coords, types, box, table=True):
    """Energy and its gradients with respect to the fitting parameters (flat,
    per model type: per layer [(win + 1) x wout] W then b, then w_out and
    b_out) and, with table=True, the table coefficients [ntypes, ntypes, n,
    6, M] (coefficients of u^q, u = s/h - k; host arrays)."""
    nf, nt = dp_param_sizes(h)
    n = int(np.shape(coords)[0])
    gf = np.zeros(nf)
    gt = np.zeros(nt) if table else None
    e = np.zeros(1)
    c, ck, _ = _ptr(coords, np.float64)  # ck, tk, bk keep the arrays alive
    t, tk, _ = _ptr(types, np.int32)
    b, bk, _ = _ptr(box, np.float64)
    _check(lib.dp_param_grad(h, n, c, t, b, e.ctypes.data_as(C.c_void_p),
                             gf.ctypes.data_as(C.c_void_p),
                             gt.ctypes.data_as(C.c_void_p) if gt is not None else None), h)
    return float(e[0]), gf, gt


def dp_get_params(h):
    """(fit [n_fit], table [n_table]) the model's current parameters (FP64
    copies of the device's FP32 values; layouts as dp_param_grad)."""
    nf, nt = dp_param_sizes(h)
    fit, tab = np.zeros(nf), np.zeros(nt)
    _check(lib.dp_get_params(h, fit.ctypes.data_as(C.c_void_p), tab.ctypes.data_as(C.c_void_p)), h)
    return fit, tab


def dp_set_params(h, fit=None, table=None):
    """Replace the fitting parameters and/or the embedding representation
    (table coefficients, or an untabulated handle's embedding nets)."""
    nf, nt = dp_param_sizes(h)
    f = np.ascontiguousarray(fit, np.float64).ravel() if fit is not None else None
    t = np.ascontiguousarray(table, np.float64).ravel() if table is not None else None
    if f is not None and f.size != nf:
        raise ValueError(f"fit has {f.size} values, the model {nf}")
    if t is not None and t.size != nt:
        raise ValueError(f"table has {t.size} values, the model {nt}")
    _check(lib.dp_set_params(h, f.ctypes.data_as(C.c_void_p) if f is not None else None,
                             t.ctypes.data_as(C.c_void_p) if t is not None else None), h)


def dp_fitting(h, types, T):
    """Per-atom energies and dE/dT for given T [n, 4, M] (host arrays)."""
    T = np.ascontiguousarray(T, np.float32)
    n = T.shape[0]
    t = np.ascontiguousarray(types, np.int32)
    e = np.zeros(max(n, 1))
    dT = np.zeros_like(T) if n else np.zeros((1,) + T.shape[1:], np.float32)
    _check(lib.dp_fitting(h, n, t.ctypes.data_as(C.c_void_p), T.ctypes.data_as(C.c_void_p),
                          e.ctypes.data_as(C.c_void_p), dT.ctypes.data_as(C.c_void_p)), h)
    return e[:n], dT[:n]
