"""ctypes front end of the FP64 CPU oracle (oracle.c) -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the CPU-baseline leg of the bench may
import this package.  The product path (the CUDA library and its binding)
never does.  The oracle shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ERRORS = {0: "ok", 1: "arg", 2: "model", 4: "nomem", 5: "sel overflow",
          6: "table range", 7: "box"}


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP, no FP contraction so that the
    results are the same on x86-64 and aarch64)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        p, i32p, i64p = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64)
        dp = C.POINTER(C.c_double)
        d, i64, i = C.c_double, C.c_int64, C.c_int
        sig = {
            "orc_set_threads": (None, [i]),
            "orc_get_threads": (i, []),
            "orc_model_load": (p, [C.c_char_p]),
            "orc_model_free": (None, [p]),
            "orc_model_dims": (i, [p, i32p]),
            "orc_switch": (None, [d, d, d, dp, dp]),
            "orc_env_row": (d, [dp, d, d, dp, dp]),
            "orc_embed": (i, [p, i, i, d, dp, dp, dp]),
            "orc_fit": (i, [p, i, dp, dp, dp]),
            "orc_set_tanh_table": (None, [i]),
            "orc_act": (d, [d, dp]),
            "orc_table_build": (p, [p, d, d]),
            "orc_table_build_ext": (p, [p, d, d, d, i]),
            "orc_table_ext": (i, [p, i32p, dp]),
            "orc_table_free": (None, [p]),
            "orc_table_dims": (i, [p, i32p, dp]),
            "orc_table_coeffs": (i, [p, i, i, dp]),
            "orc_table_eval": (i, [p, i, i, d, dp, dp]),
            "orc_hermite5": (None, [dp, dp, d, dp]),
            "orc_wrap": (d, [d, d]),
            "orc_neighbors": (i64, [i64, dp, dp, d, i, i64, i32p]),
            "orc_eval": (i, [p, p, d, d, i32p, i64, dp, i32p, dp, dp, dp, dp, dp, i64p]),
            "orc_atom_descriptor": (i, [p, p, d, d, i32p, i64, dp, i32p, dp, i64, dp, dp]),
            "orc_eval_subset": (i, [p, p, d, d, i32p, i64, dp, i32p, dp, i64, i64p, dp,
                                    i64, i64p, dp]),
            "orc_md": (i, [p, p, d, d, i32p, i64, dp, dp, dp, i, i32p, dp, dp, d, i, dp]),
            "orc_fit_param_count": (i64, [p]),
            "orc_model_fit_params": (i, [p, i, dp, dp]),
            "orc_table_set_coeffs": (i, [p, i, i, dp]),
            "orc_param_grad": (i, [p, p, d, d, i32p, i64, dp, i32p, dp, dp, dp, dp]),
            "orc_emb_param_count": (i64, [p]),
            "orc_model_emb_params": (i, [p, i, i, dp, dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i32(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _i64(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class OracleError(RuntimeError):
    def __init__(self, code, what=""):
        super().__init__(f"oracle error {code} ({ERRORS.get(code, '?')}) {what}")
        self.code = code


def set_tanh_table(on: bool) -> None:
    """Fitting-net activation: exact tanh (default) or the Sec. 3.5 table."""
    lib().orc_set_tanh_table(1 if on else 0)


def act(a: float):
    """(t, dt/da) of the fitting-net activation in the current mode."""
    dt = C.c_double()
    t = lib().orc_act(float(a), C.byref(dt))
    return t, dt.value


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return lib().orc_get_threads()


class Model:
    def __init__(self, path):
        self.path = str(path)
        self.h = lib().orc_model_load(self.path.encode())
        if not self.h:
            raise OracleError(2, self.path)
        dims = np.zeros(6, np.int32)
        lib().orc_model_dims(self.h, _i32(dims))
        self.ntypes, self.M, self.m_lt, self.din, self.d1, self.n_fit = (int(v) for v in dims)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_model_free(self.h)
            self.h = None

    def embed(self, ti, tj, s):
        g, dg, d2g = (np.zeros(self.M) for _ in range(3))
        e = lib().orc_embed(self.h, ti, tj, float(s), _d(g), _d(dg), _d(d2g))
        if e:
            raise OracleError(e)
        return g, dg, d2g

    @property
    def n_fit_params(self) -> int:
        """Length of one centre type's fitting-parameter layout (per layer k a
        [(win_k + 1), wout_k] block: W_k rows then b_k; then w_out, b_out)."""
        return int(lib().orc_fit_param_count(self.h))

    def fit_params(self, ti):
        out = np.zeros(self.n_fit_params)
        e = lib().orc_model_fit_params(self.h, ti, _d(out), None)
        if e:
            raise OracleError(e)
        return out

    def set_fit_params(self, ti, values):
        v = _f64(values)
        assert v.size == self.n_fit_params
        e = lib().orc_model_fit_params(self.h, ti, None, _d(v))
        if e:
            raise OracleError(e)

    @property
    def n_emb_params(self) -> int:
        """Length of one type pair's embedding-net parameter layout."""
        return int(lib().orc_emb_param_count(self.h))

    def emb_params(self, ti, tj):
        out = np.zeros(self.n_emb_params)
        e = lib().orc_model_emb_params(self.h, ti, tj, _d(out), None)
        if e:
            raise OracleError(e)
        return out

    def set_emb_params(self, ti, tj, values):
        v = _f64(values)
        assert v.size == self.n_emb_params
        e = lib().orc_model_emb_params(self.h, ti, tj, None, _d(v))
        if e:
            raise OracleError(e)

    def fit(self, ti, D):
        D = _f64(D)
        E = np.zeros(1)
        dD = np.zeros(self.din)
        e = lib().orc_fit(self.h, ti, _d(D), _d(E), _d(dD))
        if e:
            raise OracleError(e)
        return float(E[0]), dD


class Table:
    """Sec. 3.2 table of the model's embedding nets: intervals of width h up
    to s_max, and (s_ext > s_max) an extrapolation region of intervals of
    width ext_stride * h up to s_ext."""

    def __init__(self, model: Model, h: float, s_max: float, s_ext: float = 0.0,
                 ext_stride: int = 10):
        self.model = model
        self.h_ptr = lib().orc_table_build_ext(model.h, float(h), float(s_max), float(s_ext),
                                               int(ext_stride))
        if not self.h_ptr:
            raise OracleError(1, "table build")
        n = np.zeros(1, np.int32)
        hh = np.zeros(1)
        lib().orc_table_dims(self.h_ptr, _i32(n), _d(hh))
        self.n, self.h = int(n[0]), float(hh[0])
        lib().orc_table_ext(self.h_ptr, _i32(n), _d(hh))
        self.n_fine, self.H = int(n[0]), float(hh[0])

    def widths(self):
        """[n] interval widths (h, then H in the extrapolation region)."""
        return np.where(np.arange(self.n) < self.n_fine, self.h, self.H)

    def nodes(self):
        """[n + 1] node positions."""
        k = np.arange(self.n + 1)
        return np.where(k <= self.n_fine, k * self.h, self.n_fine * self.h + (k - self.n_fine) * self.H)

    @property
    def handle(self):
        return self.h_ptr

    def __del__(self):
        if getattr(self, "h_ptr", None) and _lib is not None:
            _lib.orc_table_free(self.h_ptr)
            self.h_ptr = None

    def coeffs(self, ti=0, tj=0):
        out = np.zeros((self.n, 6, self.model.M))
        e = lib().orc_table_coeffs(self.h_ptr, ti, tj, _d(out))
        if e:
            raise OracleError(e)
        return out

    def set_coeffs(self, ti, tj, a):
        a = _f64(a, (self.n, 6, self.model.M))
        e = lib().orc_table_set_coeffs(self.h_ptr, ti, tj, _d(a))
        if e:
            raise OracleError(e)

    def eval(self, ti, tj, s):
        g, dg = np.zeros(self.model.M), np.zeros(self.model.M)
        out = lib().orc_table_eval(self.h_ptr, ti, tj, float(s), _d(g), _d(dg))
        return g, dg, bool(out)


def hermite5(y0, y1, h):
    y0, y1 = _f64(y0), _f64(y1)
    a = np.zeros(6)
    lib().orc_hermite5(_d(y0), _d(y1), float(h), _d(a))
    return a


def switch(r, rc, rcs):
    sw, dsw = C.c_double(), C.c_double()
    lib().orc_switch(float(r), float(rc), float(rcs), C.byref(sw), C.byref(dsw))
    return sw.value, dsw.value


def env_row(d, rc, rcs):
    d = _f64(d)
    R, dR = np.zeros(4), np.zeros((4, 3))
    s = lib().orc_env_row(_d(d), float(rc), float(rcs), _d(R), _d(dR))
    return s, R, dR


def wrap(x, L):
    return lib().orc_wrap(float(x), float(L))


def neighbors(x, box, rlist, method=1):
    """Sorted int32 rows (i, j, n0, n1, n2) of all pairs closer than rlist."""
    x, box = _f64(x), _f64(box)
    n = len(x)
    cnt = lib().orc_neighbors(n, _d(x), _d(box), float(rlist), int(method), 0, None)
    if cnt < 0:
        raise OracleError(int(-cnt))
    out = np.zeros((max(cnt, 1), 5), np.int32)
    cnt2 = lib().orc_neighbors(n, _d(x), _d(box), float(rlist), int(method), cnt, _i32(out))
    assert cnt2 == cnt
    return out[:cnt]


def _sel(sel, ntypes):
    s = np.zeros(max(ntypes, 1), np.int32)
    s[:] = np.atleast_1d(np.asarray(sel, np.int32))[:ntypes] if np.ndim(sel) else int(sel)
    return s


def evaluate(model: Model, table, rc, rcs, sel, x, types, box, check=True):
    """Energy, per-atom energy, forces, virial (FP64) of the whole system."""
    x, box = _f64(x), _f64(box)
    types = np.ascontiguousarray(types, np.int32)
    n = len(x)
    sel = _sel(sel, model.ntypes)
    E = np.zeros(1)
    Ei = np.zeros(max(n, 1))
    F = np.zeros((max(n, 1), 3))
    V = np.zeros(9)
    diag = np.zeros(4, np.int64)
    code = lib().orc_eval(model.h, table.handle if table is not None else None,
                          float(rc), float(rcs), _i32(sel), n, _d(x), _i32(types), _d(box),
                          _d(E), _d(Ei), _d(F), _d(V), _i64(diag))
    if check and code:
        raise OracleError(code)
    return dict(energy=float(E[0]), atom_energy=Ei[:n], force=F[:n], virial=V.reshape(3, 3),
                max_nn=int(diag[0]), npairs=int(diag[1]), n_range=int(diag[2]),
                n_sel=int(diag[3]), status=int(code))


def atom_descriptor(model: Model, table, rc, rcs, sel, x, types, box, i):
    x, box = _f64(x), _f64(box)
    types = np.ascontiguousarray(types, np.int32)
    sel = _sel(sel, model.ntypes)
    T = np.zeros((4, model.M))
    D = np.zeros(model.din)
    code = lib().orc_atom_descriptor(model.h, table.handle if table is not None else None,
                                     float(rc), float(rcs), _i32(sel), len(x), _d(x),
                                     _i32(types), _d(box), int(i), _d(T), _d(D))
    if code:
        raise OracleError(code)
    return T, D


def eval_subset(model: Model, table, rc, rcs, sel, x, types, box, idx_e, idx_f):
    x, box = _f64(x), _f64(box)
    types = np.ascontiguousarray(types, np.int32)
    sel = _sel(sel, model.ntypes)
    idx_e = np.ascontiguousarray(idx_e, np.int64)
    idx_f = np.ascontiguousarray(idx_f, np.int64)
    e_out = np.zeros(max(len(idx_e), 1))
    f_out = np.zeros((max(len(idx_f), 1), 3))
    code = lib().orc_eval_subset(model.h, table.handle if table is not None else None,
                                 float(rc), float(rcs), _i32(sel), len(x), _d(x), _i32(types),
                                 _d(box), len(idx_e), _i64(idx_e), _d(e_out), len(idx_f),
                                 _i64(idx_f), _d(f_out))
    if code:
        raise OracleError(code)
    return e_out[:len(idx_e)], f_out[:len(idx_f)]


def md(model: Model, table, rc, rcs, sel, x, v, types, masses, box, dt, nsteps, f=None):
    """Velocity-Verlet NVE; returns (x, v, f, thermo[nsteps+1, 4]).  Passing
    the forces f at x skips the initial force evaluation."""
    x, v, box = _f64(x).copy(), _f64(v).copy(), _f64(box)
    types = np.ascontiguousarray(types, np.int32)
    masses = _f64(masses)
    sel = _sel(sel, model.ntypes)
    f_valid = f is not None
    f = _f64(f).copy() if f_valid else np.zeros_like(x)
    th = np.zeros((nsteps + 1, 4))
    code = lib().orc_md(model.h, table.handle if table is not None else None, float(rc),
                        float(rcs), _i32(sel), len(x), _d(x), _d(v), _d(f), int(f_valid),
                        _i32(types), _d(masses), _d(box), float(dt), int(nsteps), _d(th))
    if code:
        raise OracleError(code)
    return x, v, f, th


def param_grad(model: Model, table, rc, rcs, sel, x, types, box, with_table=True):
    """(E, grad_fit [ntypes, n_fit_params], grad_table or None): the energy's
    gradient with respect to the fitting parameters and the embedding
    representation: for a tabulated model the table coefficients
    [ntypes, ntypes, n, 6, M] of the normalised local variable (s - k h)/h,
    i.e. c_q = a_q h^q; for the original net (table None) its weights and
    biases [ntypes, ntypes, n_emb_params]."""
    x, box = _f64(x), _f64(box)
    types = np.ascontiguousarray(types, np.int32)
    sel = _sel(sel, model.ntypes)
    E = np.zeros(1)
    gf = np.zeros((model.ntypes, model.n_fit_params))
    gt = None
    if with_table and table is not None:
        gt = np.zeros((model.ntypes, model.ntypes, table.n, 6, model.M))
    elif with_table:
        gt = np.zeros((model.ntypes, model.ntypes, model.n_emb_params))
    code = lib().orc_param_grad(model.h, table.handle if table is not None else None,
                                float(rc), float(rcs), _i32(sel), len(x), _d(x), _i32(types),
                                _d(box), _d(E), _d(gf), _d(gt) if gt is not None else None)
    if code:
        raise OracleError(code)
    return float(E[0]), gf, gt
