"""ctypes binding of ``libweno_is.so`` (C ABI in ``include/weno_is.h``).

The functions carry the ABI's names and only marshal arguments: every step of
the computation runs in the library's CUDA kernels.  Device arrays are torch
CUDA tensors (used for device memory and streams only); host arrays are numpy
arrays or CPU tensors.  If the shared library is missing or cannot be loaded
the import raises: there is no CPU fallback.

``Solver`` wraps a context for a problem description from
``paper_1908_02464_gb300.problems``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

WENO_OK, WENO_ERR_INVALID_ARG, WENO_ERR_CUDA, WENO_ERR_NONPHYSICAL, WENO_ERR_TIMEOUT, WENO_ERR_UNSUPPORTED = range(6)
STATUS_NAMES = {0: "WENO_OK", 1: "WENO_ERR_INVALID_ARG", 2: "WENO_ERR_CUDA", 3: "WENO_ERR_NONPHYSICAL",
                4: "WENO_ERR_TIMEOUT", 5: "WENO_ERR_UNSUPPORTED"}
PRECISIONS = {"fp64": 0, "fp32": 1, "mixed": 2}


class WenoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class weno_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3),
                ("bc_state", (ctypes.c_double * 5) * 2)]


class weno_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("cfl", ctypes.c_double), ("eps", ctypes.c_double),
                ("c_lambda", ctypes.c_double), ("C_thr", ctypes.c_double), ("L_char", ctypes.c_double),
                ("alpha_thr", ctypes.c_int), ("hybrid", ctypes.c_int), ("precision", ctypes.c_int),
                ("weights", ctypes.c_int), ("splitting", ctypes.c_int)]


WEIGHTS = {"reg": 0, "is": 1, "wang": 2, "linear": 3}
SPLITTINGS = {"llf": 0, "lf": 1, "rf": 2}


class weno_batch_desc(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("n", ctypes.POINTER(ctypes.c_int)), ("lo", ctypes.POINTER(ctypes.c_double)),
                ("hi", ctypes.POINTER(ctypes.c_double)), ("t_end", ctypes.POINTER(ctypes.c_double)),
                ("bc_lo", ctypes.c_int), ("bc_hi", ctypes.c_int), ("max_steps", ctypes.c_int)]


class weno_batch2d_desc(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("nx", ctypes.POINTER(ctypes.c_int)), ("ny", ctypes.POINTER(ctypes.c_int)),
                ("lo_x", ctypes.POINTER(ctypes.c_double)), ("hi_x", ctypes.POINTER(ctypes.c_double)),
                ("lo_y", ctypes.POINTER(ctypes.c_double)), ("hi_y", ctypes.POINTER(ctypes.c_double)),
                ("t_end", ctypes.POINTER(ctypes.c_double)), ("bc_lo", ctypes.c_int * 2), ("bc_hi", ctypes.c_int * 2),
                ("max_steps", ctypes.c_int)]


_vp = ctypes.c_void_p
_ip = ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)

# ABI: name -> (restype, argtypes)
SIGNATURES = {
    "weno_default_params": (ctypes.c_int, [ctypes.POINTER(weno_params)]),
    "weno_create": (ctypes.c_int, [ctypes.POINTER(weno_grid), ctypes.POINTER(weno_params), _vp,
                                   ctypes.POINTER(_vp)]),
    "weno_destroy": (None, [_vp]),
    "weno_set_state": (ctypes.c_int, [_vp, _vp, _ip, ctypes.c_double]),
    "weno_get_state": (ctypes.c_int, [_vp, _vp, _ip, _dp]),
    "weno_rhs": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double]),
    "weno_face_flags": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _vp]),
    "weno_rhs_vjp": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double]),
    "weno_step": (ctypes.c_int, [_vp, ctypes.c_double, _dp]),
    "weno_advance": (ctypes.c_int, [_vp, ctypes.c_double, _ip, ctypes.POINTER(_ip)]),
    "weno_conserved_totals": (ctypes.c_int, [_vp, _dp]),
    "weno_weno_face_count": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_ulonglong), _ip]),
    "weno_get_time": (ctypes.c_int, [_vp, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    "weno_last_error": (ctypes.c_char_p, [_vp]),
    "weno_measure_fma_peak": (ctypes.c_int, [_ip, _dp, _dp]),
    "weno_arith_selftest": (ctypes.c_int, [_vp, ctypes.c_longlong, _vp]),
    "weno_enqueue_steps": (ctypes.c_int, [_vp, ctypes.c_double, _ip]),
    "weno_autotune": (ctypes.c_int, [_vp, _ip, ctypes.POINTER(_ip)]),
    "weno_batch_create": (ctypes.c_int, [ctypes.POINTER(weno_batch_desc), ctypes.POINTER(weno_params), _vp,
                                         ctypes.POINTER(_vp)]),
    "weno_batch2d_create": (ctypes.c_int, [ctypes.POINTER(weno_batch2d_desc), ctypes.POINTER(weno_params), _vp,
                                           ctypes.POINTER(_vp)]),
    "weno_batch_run": (ctypes.c_int, [_vp, _vp]),
    "weno_batch_results": (ctypes.c_int, [_vp, ctypes.POINTER(_ip), ctypes.POINTER(ctypes.c_longlong), _dp]),
    "weno_batch_weno_face_count": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_ulonglong), _ip]),
    "weno_batch_set_config": (ctypes.c_int, [_vp, _ip, _ip, ctypes.POINTER(ctypes.c_int)]),
    "weno_batch_autotune": (ctypes.c_int, [_vp, _vp, _ip, ctypes.POINTER(_ip)]),
    "weno_batch_destroy": (None, [_vp]),
    "weno_batch_last_error": (ctypes.c_char_p, [_vp]),
    "weno_batch_solve": (ctypes.c_int, [ctypes.POINTER(weno_batch_desc), ctypes.POINTER(weno_params), _vp, _vp,
                                        ctypes.POINTER(_ip)]),
    "weno_set_tiles": (ctypes.c_int, [_vp, ctypes.POINTER(_ip)]),
    "weno_conserved_totals_noalloc": (ctypes.c_int, [_ip, ctypes.POINTER(_ip), _dp, _ip, _vp, _vp, _vp]),
    "weno_time_sweeps": (ctypes.c_int, [_vp, _ip, _vp, ctypes.c_size_t, _dp, ctypes.POINTER(ctypes.c_ulonglong)]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load the shared library (building it in-tree if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libweno_is.so not found at {_build.LIB}; run paper_1908_02464_gb300.build")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st: int, ctx=None):
    if st != WENO_OK:
        msg = load().weno_last_error(ctx)
        raise WenoError(st, msg.decode() if msg else "")


def _ptr(x) -> int:
    """Address of a torch tensor or numpy array (must be contiguous)."""
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    assert isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]
    return x.ctypes.data


def _on_device(x) -> int:
    return int(hasattr(x, "is_cuda") and x.is_cuda)


# ----------------------------------------------------------------- ABI names

def weno_default_params() -> weno_params:
    p = weno_params()
    _check(load().weno_default_params(ctypes.byref(p)))
    return p


def weno_create(grid: weno_grid, params: weno_params, stream: int = 0) -> int:
    ctx = _vp()
    _check(load().weno_create(ctypes.byref(grid), ctypes.byref(params), _vp(stream or None), ctypes.byref(ctx)))
    return ctx.value


def weno_destroy(ctx: int) -> None:
    load().weno_destroy(_vp(ctx))


def weno_set_state(ctx: int, U, t: float = 0.0) -> None:
    _check(load().weno_set_state(_vp(ctx), _vp(_ptr(U)), _on_device(U), float(t)), _vp(ctx))


def weno_get_state(ctx: int, out) -> float:
    t = ctypes.c_double(0.0)
    _check(load().weno_get_state(_vp(ctx), _vp(_ptr(out)), _on_device(out), ctypes.byref(t)), _vp(ctx))
    return t.value


def weno_rhs(ctx: int, U_dev, dUdt_dev, t: float = 0.0) -> None:
    _check(load().weno_rhs(_vp(ctx), _vp(_ptr(U_dev)), _vp(_ptr(dUdt_dev)), float(t)), _vp(ctx))


def weno_rhs_vjp(ctx: int, U_dev, w_dev, gU_dev, t: float = 0.0) -> None:
    _check(load().weno_rhs_vjp(_vp(ctx), _vp(_ptr(U_dev)), _vp(_ptr(w_dev)), _vp(_ptr(gU_dev)), float(t)), _vp(ctx))


def weno_face_flags(ctx: int, U_dev, t: float, flags_dev) -> None:
    _check(load().weno_face_flags(_vp(ctx), _vp(_ptr(U_dev)), float(t), _vp(_ptr(flags_dev))), _vp(ctx))


def weno_step(ctx: int, t_end: float) -> float:
    dt = ctypes.c_double(0.0)
    _check(load().weno_step(_vp(ctx), float(t_end), ctypes.byref(dt)), _vp(ctx))
    return dt.value


def weno_advance(ctx: int, t_end: float, max_steps: int) -> int:
    k = ctypes.c_int(0)
    _check(load().weno_advance(_vp(ctx), float(t_end), int(max_steps), ctypes.byref(k)), _vp(ctx))
    return k.value


def weno_conserved_totals(ctx: int, nvar: int) -> np.ndarray:
    out = np.zeros(nvar)
    _check(load().weno_conserved_totals(_vp(ctx), out.ctypes.data_as(_dp)), _vp(ctx))
    return out


def weno_weno_face_count(ctx: int, reset: bool = False) -> int:
    c = ctypes.c_ulonglong(0)
    _check(load().weno_weno_face_count(_vp(ctx), ctypes.byref(c), int(reset)), _vp(ctx))
    return c.value


def weno_get_time(ctx: int):
    t = ctypes.c_double(0.0)
    s = ctypes.c_longlong(0)
    _check(load().weno_get_time(_vp(ctx), ctypes.byref(t), ctypes.byref(s)), _vp(ctx))
    return t.value, s.value


def weno_measure_fma_peak(precision: int = 0):
    f = ctypes.c_double(0.0)
    s = ctypes.c_double(0.0)
    _check(load().weno_measure_fma_peak(int(precision), ctypes.byref(f), ctypes.byref(s)))
    return f.value, s.value


def weno_arith_selftest(x_dev):
    """[rcp_newton(x), 1/x, rsqrt_refined(x), rsqrt(x)] of a float64 CUDA
    tensor as a (4, n) float64 CUDA tensor (diagnostic of the sweep
    arithmetic)."""
    import torch
    x = x_dev.contiguous()
    out = torch.empty((4, x.numel()), dtype=torch.float64, device=x.device)
    _check(load().weno_arith_selftest(_vp(_ptr(x)), int(x.numel()), _vp(_ptr(out))))
    return out


def weno_conserved_totals_noalloc(dim: int, n, dx, precision: str, U_dev, totals_dev, stream: int = 0) -> None:
    """Totals of a caller-owned device state into a caller-owned device buffer,
    with no allocation (see include/weno_is.h)."""
    nn = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    dd = (ctypes.c_double * 3)(*(list(dx) + [1.0] * (3 - len(dx))))
    _check(load().weno_conserved_totals_noalloc(int(dim), nn, dd, PRECISIONS[precision], _vp(_ptr(U_dev)),
                                                _vp(_ptr(totals_dev)), _vp(stream or None)))


def weno_autotune(ctx: int, reps: int = 3):
    v = (ctypes.c_int * 3)()
    _check(load().weno_autotune(_vp(ctx), int(reps), v), _vp(ctx))
    return list(v)


def weno_set_tiles(ctx: int, variants) -> None:
    v = (ctypes.c_int * 3)(*(list(variants) + [0] * (3 - len(variants))))
    _check(load().weno_set_tiles(_vp(ctx), v), _vp(ctx))


def weno_enqueue_steps(ctx: int, t_end: float, nsteps: int) -> None:
    _check(load().weno_enqueue_steps(_vp(ctx), float(t_end), int(nsteps)), _vp(ctx))


def weno_time_sweeps(ctx: int, dim: int, reps: int, flush=None):
    ms = (ctypes.c_double * 3)()
    wf = (ctypes.c_ulonglong * 3)()
    fp = _vp(_ptr(flush)) if flush is not None else None
    fb = flush.numel() * flush.element_size() if flush is not None else 0
    _check(load().weno_time_sweeps(_vp(ctx), int(reps), fp, fb, ms, wf), _vp(ctx))
    return list(ms)[:dim], list(wf)[:dim]


# ----------------------------------------------------------------- helpers

def make_grid(problem: dict) -> weno_grid:
    g = weno_grid()
    dim = problem["dim"]
    if dim not in (1, 2, 3):
        raise ValueError("the CUDA library solves the Euler equations in 1, 2 or 3 dimensions")
    g.dim = dim
    for a in range(3):
        g.n[a] = int(problem["n"][a]) if a < dim else 1
        g.lo[a] = float(problem["lo"][a]) if a < dim else 0.0
        g.hi[a] = float(problem["hi"][a]) if a < dim else 1.0
        g.bc_lo[a] = int(problem["bc_lo"][a]) if a < dim else 0
        g.bc_hi[a] = int(problem["bc_hi"][a]) if a < dim else 0
    bs = problem.get("bc_state", [[0.0] * 5, [0.0] * 5])
    for s in range(2):
        for v in range(5):
            g.bc_state[s][v] = float(bs[s][v]) if v < len(bs[s]) else 0.0
    return g


def make_params(problem: dict, precision: str = "fp64") -> weno_params:
    p = weno_default_params()
    for k in ("gamma", "cfl", "eps", "c_lambda", "C_thr", "L_char"):
        if k in problem:
            setattr(p, k, float(problem[k]))
    if "alpha_thr" in problem:
        p.alpha_thr = int(problem["alpha_thr"])
    if "hybrid" in problem:
        p.hybrid = int(problem["hybrid"])
    p.weights = WEIGHTS[problem.get("weights", "reg")]
    p.splitting = SPLITTINGS[problem.get("splitting", "llf")]
    p.precision = PRECISIONS[precision]
    return p


class Solver:
    """A context for one problem: state, RHS, steps (all on the GPU)."""

    def __init__(self, problem: dict, precision: str = "fp64", stream=None):
        import torch
        self.problem = problem
        self.precision = precision
        self.dim = problem["dim"]
        self.nvar = self.dim + 2
        self.shape = (self.nvar,) + tuple(reversed([int(m) for m in problem["n"][:self.dim]]))
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.np_dtype = np.float64 if precision == "fp64" else np.float32
        s = stream.cuda_stream if stream is not None else 0
        self.ctx = weno_create(make_grid(problem), make_params(problem, precision), s)

    def close(self):
        if self.ctx:
            weno_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n_faces(self) -> int:
        n = list(self.shape[1:])[::-1]
        tot = 0
        for a in range(self.dim):
            m = list(n)
            m[a] += 1
            tot += int(np.prod(m))
        return tot

    def set_state(self, U, t: float = 0.0):
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=self.np_dtype)
        else:
            U = U.to(self.dtype).contiguous()
        assert tuple(U.shape) == self.shape, (U.shape, self.shape)
        weno_set_state(self.ctx, U, t)

    def get_state(self, device: bool = False):
        import torch
        if device:
            out = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        else:
            out = np.empty(self.shape, dtype=self.np_dtype)
        t = weno_get_state(self.ctx, out)
        return out, t

    def rhs(self, U_dev, t: float = 0.0, out=None):
        import torch
        U_dev = U_dev.to(self.dtype).contiguous()
        if out is None:
            out = torch.empty_like(U_dev)
        weno_rhs(self.ctx, U_dev, out, t)
        return out

    def rhs_vjp(self, U_dev, w_dev, t: float = 0.0, out=None):
        """(d RHS / d U)^T w at U (flags and LLF argmax held fixed)."""
        import torch
        U_dev = U_dev.to(self.dtype).contiguous()
        w_dev = w_dev.to(self.dtype).contiguous()
        if out is None:
            out = torch.empty_like(U_dev)
        weno_rhs_vjp(self.ctx, U_dev, w_dev, out, t)
        return out

    def face_flags(self, U_dev, t: float = 0.0):
        import torch
        U_dev = U_dev.to(self.dtype).contiguous()
        flags = torch.full((self.n_faces(),), 255, dtype=torch.uint8, device=U_dev.device)
        weno_face_flags(self.ctx, U_dev, t, flags)
        return flags

    def step(self, t_end: float) -> float:
        return weno_step(self.ctx, t_end)

    def advance(self, t_end: float, max_steps: int = 2 ** 31 - 1) -> int:
        return weno_advance(self.ctx, t_end, max_steps)

    def totals(self) -> np.ndarray:
        return weno_conserved_totals(self.ctx, self.nvar)

    def weno_faces(self, reset: bool = False) -> int:
        return weno_weno_face_count(self.ctx, reset)

    def time(self):
        return weno_get_time(self.ctx)

    def enqueue_steps(self, t_end: float, nsteps: int):
        weno_enqueue_steps(self.ctx, t_end, nsteps)

    def set_tiles(self, variants):
        weno_set_tiles(self.ctx, variants)

    def autotune(self, reps: int = 3):
        return weno_autotune(self.ctx, reps)[:self.dim]

    def time_sweeps(self, reps: int = 5, flush=None):
        return weno_time_sweeps(self.ctx, self.dim, reps, flush)


# ----------------------------------------------------------------- batches

def _bcheck(st: int, batch=None):
    if st != WENO_OK:
        msg = load().weno_batch_last_error(batch)
        raise WenoError(st, msg.decode() if msg else "")


def _batch_desc(N, lo, hi, t_end, bc_lo=0, bc_hi=0, max_steps=0):
    N = np.ascontiguousarray(N, dtype=np.int32)
    lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, dtype=np.float64), N.shape))
    hi = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, dtype=np.float64), N.shape))
    te = np.ascontiguousarray(t_end, dtype=np.float64)
    d = weno_batch_desc()
    d.count = int(N.size)
    d.n = N.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    d.lo = lo.ctypes.data_as(_dp)
    d.hi = hi.ctypes.data_as(_dp)
    d.t_end = te.ctypes.data_as(_dp)
    d.bc_lo, d.bc_hi, d.max_steps = int(bc_lo), int(bc_hi), int(max_steps)
    return d, (N, lo, hi, te)


def weno_batch_create(N, lo, hi, t_end, params: weno_params, bc_lo=0, bc_hi=0, max_steps=0, stream: int = 0) -> int:
    d, keep = _batch_desc(N, lo, hi, t_end, bc_lo, bc_hi, max_steps)
    b = _vp()
    _bcheck(load().weno_batch_create(ctypes.byref(d), ctypes.byref(params), _vp(stream or None), ctypes.byref(b)))
    return b.value


def weno_batch2d_create(NX, NY, lo, hi, t_end, params: weno_params, bc_lo=(0, 0), bc_hi=(0, 0), max_steps=0,
                        stream: int = 0) -> int:
    """lo, hi: (x, y) pairs, one for all instances or one per instance."""
    NX = np.ascontiguousarray(NX, dtype=np.int32)
    NY = np.ascontiguousarray(NY, dtype=np.int32)
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), NX.shape + (2,))
    hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), NX.shape + (2,))
    cols = [np.ascontiguousarray(a[:, k]) for a in (lo, hi) for k in (0, 1)]
    te = np.ascontiguousarray(t_end, dtype=np.float64)
    d = weno_batch2d_desc()
    d.count = int(NX.size)
    d.nx = NX.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    d.ny = NY.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    d.lo_x, d.lo_y, d.hi_x, d.hi_y = (c.ctypes.data_as(_dp) for c in cols)
    d.t_end = te.ctypes.data_as(_dp)
    for k in range(2):
        d.bc_lo[k], d.bc_hi[k] = int(bc_lo[k]), int(bc_hi[k])
    d.max_steps = int(max_steps)
    b = _vp()
    _bcheck(load().weno_batch2d_create(ctypes.byref(d), ctypes.byref(params), _vp(stream or None), ctypes.byref(b)))
    return b.value


def weno_batch_run(batch: int, U_dev) -> None:
    _bcheck(load().weno_batch_run(_vp(batch), _vp(_ptr(U_dev))), _vp(batch))


def weno_batch_results(batch: int, count: int, raise_on_failure: bool = False):
    st = np.zeros(count, dtype=np.int32)
    steps = np.zeros(count, dtype=np.int64)
    t = np.zeros(count)
    r = load().weno_batch_results(_vp(batch), st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  steps.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), t.ctypes.data_as(_dp))
    if r != WENO_OK and (raise_on_failure or r != WENO_ERR_NONPHYSICAL):
        _bcheck(r, _vp(batch))
    return st, steps, t


def weno_batch_autotune(batch: int, U_dev, trial_steps: int = 4):
    c = (ctypes.c_int * 2)()
    _bcheck(load().weno_batch_autotune(_vp(batch), _vp(_ptr(U_dev)), int(trial_steps), c), _vp(batch))
    return list(c)


def weno_batch_destroy(batch: int) -> None:
    load().weno_batch_destroy(_vp(batch))


def weno_batch_solve(N, lo, hi, t_end, params: weno_params, U_dev, bc_lo=0, bc_hi=0, max_steps=0, stream: int = 0):
    d, keep = _batch_desc(N, lo, hi, t_end, bc_lo, bc_hi, max_steps)
    st = np.zeros(d.count, dtype=np.int32)
    r = load().weno_batch_solve(ctypes.byref(d), ctypes.byref(params), _vp(stream or None), _vp(_ptr(U_dev)),
                                st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if r not in (WENO_OK, WENO_ERR_NONPHYSICAL):
        _bcheck(r)
    return st


class Batch:
    """Many independent 1D Euler problems solved by one persistent launch."""

    def __init__(self, N, lo, hi, t_end, precision: str = "fp64", gamma: float = 1.4, bc=(0, 0),
                 max_steps: int = 0, stream=None, **params):
        import torch
        self.N = np.asarray(N, dtype=np.int64)
        self.count = int(self.N.size)
        self.offsets = np.concatenate([[0], np.cumsum(3 * self.N)])
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        p = weno_default_params()
        p.gamma = gamma
        for k, v in params.items():
            setattr(p, k, v)
        p.precision = PRECISIONS[precision]
        s = stream.cuda_stream if stream is not None else 0
        self.handle = weno_batch_create(self.N, lo, hi, t_end, p, bc[0], bc[1], max_steps, s)

    def pack(self, states):
        """Device array holding the states ([3][n_i] each) back to back."""
        import torch
        flat = np.concatenate([np.asarray(u, dtype=np.float64).reshape(-1) for u in states])
        return torch.from_numpy(flat).to("cuda", self.dtype)

    def unpack(self, U_dev):
        h = U_dev.double().cpu().numpy()
        return [h[self.offsets[i]:self.offsets[i + 1]].reshape(3, -1) for i in range(self.count)]

    def run(self, U_dev):
        weno_batch_run(self.handle, U_dev)

    def results(self):
        return weno_batch_results(self.handle, self.count)

    def autotune(self, U_dev, trial_steps: int = 4):
        return weno_batch_autotune(self.handle, U_dev, trial_steps)

    def set_config(self, variant: int, blocks_per_sm: int = 0) -> int:
        """Fix the tile variant and residency without timing; returns the CTAs a run launches."""
        b = ctypes.c_int(0)
        _bcheck(load().weno_batch_set_config(self.handle, int(variant), int(blocks_per_sm), ctypes.byref(b)),
                self.handle)
        return b.value

    def weno_faces(self, reset: bool = False) -> int:
        c = ctypes.c_ulonglong(0)
        _bcheck(load().weno_batch_weno_face_count(self.handle, ctypes.byref(c), int(reset)), self.handle)
        return c.value

    def close(self):
        if self.handle:
            weno_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch2D(Batch):
    """Many independent 2D Euler problems (instance i: NY[i] x NX[i] cells,
    state [4][NY[i]][NX[i]]) solved by one persistent launch."""

    def __init__(self, NX, NY, lo, hi, t_end, precision: str = "fp64", gamma: float = 1.4, bc_lo=(0, 0),
                 bc_hi=(0, 0), max_steps: int = 0, stream=None, **params):
        import torch
        self.NX = np.asarray(NX, dtype=np.int64)
        self.NY = np.asarray(NY, dtype=np.int64)
        self.count = int(self.NX.size)
        self.offsets = np.concatenate([[0], np.cumsum(4 * self.NX * self.NY)])
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        p = weno_default_params()
        p.gamma = gamma
        for k, v in params.items():
            setattr(p, k, v)
        p.precision = PRECISIONS[precision]
        s = stream.cuda_stream if stream is not None else 0
        self.handle = weno_batch2d_create(self.NX, self.NY, lo, hi, t_end, p, bc_lo, bc_hi, max_steps, s)

    def unpack(self, U_dev):
        h = U_dev.double().cpu().numpy()
        return [h[self.offsets[i]:self.offsets[i + 1]].reshape(4, int(self.NY[i]), int(self.NX[i]))
                for i in range(self.count)]


# ----------------------------------------------------------------- autograd

def _make_rhs_function():
    import torch

    class RhsFunction(torch.autograd.Function):
        """dU/dt = RHS(U) with a hand-written backward (weno_rhs_vjp): the
        backward pass recomputes the nonlinear weights instead of storing
        them."""

        @staticmethod
        def forward(ctx, U, solver, t):
            ctx.solver = solver
            ctx.t = float(t)
            ctx.save_for_backward(U)
            return solver.rhs(U.detach(), t)

        @staticmethod
        def backward(ctx, grad_out):
            (U,) = ctx.saved_tensors
            g = ctx.solver.rhs_vjp(U.detach(), grad_out.contiguous(), ctx.t)
            return g.to(U.dtype), None, None

    return RhsFunction


_RhsFunction = None


def rhs_autograd(solver: "Solver", U, t: float = 0.0):
    """Differentiable semi-discrete operator for torch autograd."""
    global _RhsFunction
    if _RhsFunction is None:
        _RhsFunction = _make_rhs_function()
    return _RhsFunction.apply(U, solver, t)
