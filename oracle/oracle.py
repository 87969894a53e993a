"""ctypes front-end of the FP64 CPU oracle (``weno_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  Nothing in the library
package imports this module; the oracle shares no code with the CUDA path.

The oracle is plain FP64 C++ written step by step from the paper (Zhu & Hu,
arXiv 1908.02464): Eq. eq6, eq11, eq18, eq8-r for the scalar reconstruction,
Sec. 2.4 steps (1)-(6) for the characteristic flux, Eq. eq27-29 for the
detector and regularization parameter, Eq. eqhy / linearupwind / eq31 for the
hybrid switch, and the third-order TVD Runge-Kutta scheme of Sec. 4.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "weno_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

BC_TRANSMISSIVE, BC_REFLECT, BC_PERIODIC, BC_INFLOW, BC_DMR_BOTTOM, BC_DMR_TOP, BC_JET = range(7)
WEIGHTS = {"reg": 0, "is": 1, "wang": 2, "linear": 3}
SPLITTING = {"llf": 0, "lf": 1, "rf": 2}


class OrCfg(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("bc_lo", ctypes.c_int * 3),
        ("bc_hi", ctypes.c_int * 3),
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("c_lambda", ctypes.c_double),
        ("C_thr", ctypes.c_double),
        ("L_char", ctypes.c_double),
        ("alpha_thr", ctypes.c_int),
        ("hybrid", ctypes.c_int),
        ("weights", ctypes.c_int),
        ("splitting", ctypes.c_int),
        ("bc_state", (ctypes.c_double * 5) * 2),
        ("adv_speed", ctypes.c_double),
        ("dt_fixed", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (no CUDA involved)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            cp = ctypes.POINTER(OrCfg)
            L.or_recon.restype = ctypes.c_double
            L.or_recon.argtypes = [dp, ctypes.c_double, ctypes.c_int, ctypes.c_double, dp]
            L.or_roe_eigen.argtypes = [cp, ctypes.c_int, dp, dp, dp, dp, dp, dp]
            L.or_cell_flux.argtypes = [cp, ctypes.c_int, dp, dp, dp]
            L.or_face_flux.restype = ctypes.c_int
            L.or_face_flux.argtypes = [cp, ctypes.c_int, ctypes.c_double, dp, dp, dp, dp]
            L.or_eps_h.restype = ctypes.c_double
            L.or_eps_h.argtypes = [cp, ctypes.c_double]
            L.or_fill_ghosts.argtypes = [cp, ctypes.c_double, dp, dp]
            L.or_rhs.argtypes = [cp, ctypes.c_double, dp, dp, ctypes.POINTER(ctypes.c_ubyte), dp]
            L.or_rhs_jvp.argtypes = [cp, ctypes.c_double, dp, dp, dp, dp]
            L.or_cfl_dt.restype = ctypes.c_double
            L.or_cfl_dt.argtypes = [cp, dp]
            L.or_step.restype = ctypes.c_int
            L.or_step.argtypes = [cp, dp, dp, ctypes.c_double, dp]
            L.or_advance.restype = ctypes.c_int
            L.or_advance.argtypes = [cp, dp, dp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            L.or_totals.argtypes = [cp, dp, dp]
            ll = ctypes.POINTER(ctypes.c_longlong)
            L.or_count_cell.argtypes = [cp, ctypes.c_int, dp, ll]
            L.or_count_face.restype = ctypes.c_int
            L.or_count_face.argtypes = [cp, ctypes.c_int, ctypes.c_double, dp, ll]
            L.or_riemann_star.restype = ctypes.c_int
            L.or_riemann_star.argtypes = [ctypes.c_double, dp, dp, dp, dp]
            L.or_riemann_sample.restype = ctypes.c_int
            L.or_riemann_sample.argtypes = [ctypes.c_double, dp, dp, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int, dp, dp]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_cfg(problem: dict) -> OrCfg:
    """Translate a problem description (see ``paper_1908_02464_gb300.problems``)
    into the oracle's configuration structure."""
    c = OrCfg()
    dim = problem["dim"]
    c.dim = dim
    n = list(problem["n"]) + [1] * (3 - len(problem["n"]))
    lo = list(problem["lo"]) + [0.0] * (3 - len(problem["lo"]))
    hi = list(problem["hi"]) + [1.0] * (3 - len(problem["hi"]))
    bl = list(problem["bc_lo"]) + [0] * (3 - len(problem["bc_lo"]))
    bh = list(problem["bc_hi"]) + [0] * (3 - len(problem["bc_hi"]))
    for a in range(3):
        c.n[a] = int(n[a]); c.lo[a] = float(lo[a]); c.hi[a] = float(hi[a])
        c.bc_lo[a] = int(bl[a]); c.bc_hi[a] = int(bh[a])
    c.gamma = float(problem.get("gamma", 1.4))
    c.cfl = float(problem.get("cfl", 0.5))
    c.eps = float(problem.get("eps", 1e-20))
    c.c_lambda = float(problem.get("c_lambda", 1.0))
    c.C_thr = float(problem.get("C_thr", 1.0))
    c.L_char = float(problem.get("L_char", 1.0))
    c.alpha_thr = int(problem.get("alpha_thr", 3))
    c.hybrid = int(problem.get("hybrid", 1))
    c.weights = WEIGHTS[problem.get("weights", "reg")]
    c.splitting = SPLITTING[problem.get("splitting", "llf")]
    bs = problem.get("bc_state", [[0.0] * 5, [0.0] * 5])
    for s in range(2):
        for v in range(5):
            c.bc_state[s][v] = float(bs[s][v]) if v < len(bs[s]) else 0.0
    c.adv_speed = float(problem.get("adv_speed", 1.0))
    c.dt_fixed = float(problem.get("dt_fixed", 0.0))
    return c


def nvar(problem: dict) -> int:
    return 1 if problem["dim"] == 0 else problem["dim"] + 2


def n_faces(problem: dict) -> int:
    """Total number of faces over all swept directions."""
    dim = max(problem["dim"], 1)
    n = list(problem["n"])[:dim]
    tot = 0
    for a in range(dim):
        m = list(n)
        m[a] += 1
        tot += int(np.prod(m))
    return tot


def recon(f, lam: float, weights: str = "reg", eps: float = 1e-20):
    """Reconstruction at x_{j+1/2} from f_{j-2..j+2}; returns (fhat, detail)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    det = np.zeros(21)
    r = lib().or_recon(_dp(f), lam, WEIGHTS[weights], eps, _dp(det))
    d = {"q": det[0:4].copy(), "beta": det[4:8].copy(), "E": det[8:12].copy(),
         "tau5": det[12], "alpha": det[13:17].copy(), "omega": det[17:21].copy()}
    return r, d


def roe_eigen(problem: dict, d: int, UA, UB):
    c = make_cfg(problem)
    nv = nvar(problem)
    UA = np.ascontiguousarray(UA, dtype=np.float64)
    UB = np.ascontiguousarray(UB, dtype=np.float64)
    L = np.zeros((nv, nv)); R = np.zeros((nv, nv)); lam = np.zeros(nv); rt = np.zeros(1)
    lib().or_roe_eigen(ctypes.byref(c), d, _dp(UA), _dp(UB), _dp(L), _dp(R), _dp(lam), _dp(rt))
    return L, R, lam, rt[0]


def cell_flux(problem: dict, d: int, U):
    c = make_cfg(problem)
    nv = nvar(problem)
    U = np.ascontiguousarray(U, dtype=np.float64)
    F = np.zeros(nv); lam = np.zeros(nv)
    lib().or_cell_flux(ctypes.byref(c), d, _dp(U), _dp(F), _dp(lam))
    return F, lam


def face_flux(problem: dict, d: int, U6, eps_h: float | None = None, alpha_global=None):
    c = make_cfg(problem)
    nv = nvar(problem)
    U6 = np.ascontiguousarray(U6, dtype=np.float64).reshape(6, nv)
    if eps_h is None:
        dx = (problem["hi"][d] - problem["lo"][d]) / problem["n"][d]
        eps_h = lib().or_eps_h(ctypes.byref(c), dx)
    F = np.zeros(nv); sig = np.zeros(nv)
    ag = None
    if alpha_global is not None:
        ag = np.ascontiguousarray(alpha_global, dtype=np.float64)
    smooth = lib().or_face_flux(ctypes.byref(c), d, eps_h, _dp(U6), _dp(ag) if ag is not None else None,
                                _dp(F), _dp(sig))
    return F, bool(smooth), sig


def eps_h(problem: dict, d: int = 0) -> float:
    c = make_cfg(problem)
    dx = (problem["hi"][d] - problem["lo"][d]) / problem["n"][d]
    return lib().or_eps_h(ctypes.byref(c), dx)


def fill_ghosts(problem: dict, U: np.ndarray, t: float = 0.0) -> np.ndarray:
    c = make_cfg(problem)
    dim = max(problem["dim"], 1)
    n = list(problem["n"])[:dim]
    shape = [nvar(problem)] + [m + 6 for m in reversed(n)]
    Ug = np.zeros(shape)
    U = np.ascontiguousarray(U, dtype=np.float64)
    lib().or_fill_ghosts(ctypes.byref(c), t, _dp(U), _dp(Ug))
    return Ug


def rhs(problem: dict, U: np.ndarray, t: float = 0.0, want_flags: bool = False):
    """dU/dt of Eq. goveq5 (summed over directions).  U: [nvar, (nz,) (ny,) nx]."""
    c = make_cfg(problem)
    U = np.ascontiguousarray(U, dtype=np.float64)
    dU = np.zeros_like(U)
    if want_flags:
        nf = n_faces(problem)
        flags = np.zeros(nf, dtype=np.uint8)
        ratio = np.zeros(nf)
        lib().or_rhs(ctypes.byref(c), t, _dp(U), _dp(dU),
                     flags.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), _dp(ratio))
        return dU, flags, ratio
    lib().or_rhs(ctypes.byref(c), t, _dp(U), _dp(dU), None, None)
    return dU


def rhs_jvp(problem: dict, U: np.ndarray, V: np.ndarray, t: float = 0.0):
    """(dU/dt, J V): the RHS and its directional derivative along V, with the
    hybrid flags and LLF maxima held at their values for U (LLF only)."""
    assert problem.get("splitting", "llf") == "llf"
    c = make_cfg(problem)
    U = np.ascontiguousarray(U, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    dU = np.zeros_like(U)
    JV = np.zeros_like(U)
    lib().or_rhs_jvp(ctypes.byref(c), t, _dp(U), _dp(V), _dp(dU), _dp(JV))
    return dU, JV


def cfl_dt(problem: dict, U: np.ndarray) -> float:
    c = make_cfg(problem)
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().or_cfl_dt(ctypes.byref(c), _dp(U))


def step(problem: dict, U: np.ndarray, t: float, t_end: float):
    """One RK3 step in place.  Returns (status, t, dt)."""
    c = make_cfg(problem)
    assert U.dtype == np.float64 and U.flags["C_CONTIGUOUS"]
    tt = np.array([t]); dt = np.zeros(1)
    st = lib().or_step(ctypes.byref(c), _dp(U), _dp(tt), t_end, _dp(dt))
    return st, float(tt[0]), float(dt[0])


def advance(problem: dict, U: np.ndarray, t: float, t_end: float, max_steps: int = 10 ** 9):
    """Advance in place to t_end.  Returns (status, t, steps)."""
    c = make_cfg(problem)
    assert U.dtype == np.float64 and U.flags["C_CONTIGUOUS"]
    tt = np.array([t]); k = ctypes.c_int(0)
    st = lib().or_advance(ctypes.byref(c), _dp(U), _dp(tt), t_end, int(max_steps), ctypes.byref(k))
    return st, float(tt[0]), k.value


def totals(problem: dict, U: np.ndarray) -> np.ndarray:
    c = make_cfg(problem)
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.zeros(nvar(problem))
    lib().or_totals(ctypes.byref(c), _dp(U), _dp(out))
    return out


def count_cell(problem: dict, d: int, U, essential: bool = False) -> np.ndarray:
    """(add/sub, mul, div, sqrt) of one cell's quantities as written, or with
    essential=True without operations folded between known constants and
    without products / sums / quotients with structural 0 or +-1."""
    c = make_cfg(problem)
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = (ctypes.c_longlong * 8)()
    lib().or_count_cell(ctypes.byref(c), d, _dp(U), out)
    out = np.array(list(out))
    return out[4:] if essential else out[:4]


def count_face(problem: dict, d: int, U6, eps_h: float, essential: bool = False):
    """Operation counts of one face (see count_cell) and its smooth flag."""
    c = make_cfg(problem)
    U6 = np.ascontiguousarray(U6, dtype=np.float64)
    out = (ctypes.c_longlong * 8)()
    smooth = lib().or_count_face(ctypes.byref(c), d, eps_h, _dp(U6), out)
    out = np.array(list(out))
    return (out[4:] if essential else out[:4]), bool(smooth)


def riemann_star(gamma: float, WL, WR):
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    ps = np.zeros(1); us = np.zeros(1)
    vac = lib().or_riemann_star(gamma, _dp(WL), _dp(WR), _dp(ps), _dp(us))
    return bool(vac), float(ps[0]), float(us[0])


def riemann_sample(gamma: float, WL, WR, x0: float, t: float, x) -> np.ndarray:
    """Exact solution (rho, u, p) at points x and time t; interface at x0."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    W = np.zeros((3, x.size))
    vac = lib().or_riemann_sample(gamma, _dp(WL), _dp(WR), x0, t, x.size, _dp(x), _dp(W))
    if vac:
        raise ValueError("Riemann data generate vacuum")
    return W
