"""Accounting of the parity bars used by the GPU tests.

Every comparison of a CUDA result with the oracle goes through `bar()`,
which applies three levels in turn and records which one the comparison
needed:

1. "strict": per conserved variable, max |gpu - oracle| <= 1e-12
   max |oracle| (the RHS bar of the specification, normwise relative);
2. "terms": max |gpu - oracle| <= 1e-12 T_v, where T_v is the size of the
   terms whose difference the RHS is, T_v = max_cells sum_d 2 |F_v,d(U)| /
   dx_d (see `term_scale`).  The RHS of Eq. goveq5 is a difference of face
   fluxes of size |F| divided by dx; a rounding of relative size e in the
   fluxes moves it by e T_v, however small the difference itself is (a
   density RHS that vanishes analytically, momentum fluxes of 100 with an
   O(0.1) divergence);
3. "kappa": the oracle's own sensitivity kappa (how far its result moves,
   relative to max |oracle|, when its input is perturbed by one ulp at
   random) sets the bar at 10 kappa.  This is the conditioning of the
   method itself on WENO faces of quiet fields (Eq. eq8-r with eps = 1e-20:
   the weights depend on rounding noise in the detector).  The bar is capped:
   10 kappa above `cap` (KAPPA_CAP unless a test names its own cap, with its
   reason) fails the test.

Each record also holds the number of hybrid flags that differ from the
oracle's (all within FLAG_WINDOW of the threshold) and the largest
|sigma / eps_h - 1| among them.  `pytest` prints every record above level 1
at the end of the run; with the environment variable WENO_PARITY_LOG set to
a path, all records are written there as JSON lines.
"""
from __future__ import annotations

import json
import os

import numpy as np

KAPPA_CAP = 1e-9          # loosest relative bar the fallback may reach
FLAG_WINDOW = 1e-9        # |sigma / eps_h - 1| below which a flag may differ
RECORDS: list[dict] = []


def _test_id() -> str:
    return os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]


def term_scale(prob: dict, U: np.ndarray) -> np.ndarray:
    """T_v = max over cells of sum_d 2 |F_v,d(U)| / dx_d per conserved
    variable: the physical fluxes of the governing equations (Eq. goveq4 and
    its multi-D form) stand for the face fluxes they are reconstructed from."""
    dim = prob["dim"]
    U = np.asarray(U, dtype=np.float64)
    if dim == 0:
        dx = (prob["hi"][0] - prob["lo"][0]) / prob["n"][0]
        return np.array([2.0 * abs(prob.get("adv_speed", 1.0)) * np.max(np.abs(U[0])) / dx])
    g = prob.get("gamma", 1.4)
    rho = U[0]
    vel = [U[1 + d] / rho for d in range(dim)]
    p = (g - 1.0) * (U[dim + 1] - 0.5 * sum(U[1 + d] * vel[d] for d in range(dim)))
    T = np.zeros((dim + 2,) + rho.shape)
    for d in range(dim):
        dx = (prob["hi"][d] - prob["lo"][d]) / prob["n"][d]
        F = [U[1 + d]] + [U[1 + k] * vel[d] + (p if k == d else 0.0) for k in range(dim)] + \
            [(U[dim + 1] + p) * vel[d]]
        for v in range(dim + 2):
            T[v] += 2.0 * np.abs(F[v]) / dx
    return T.reshape(dim + 2, -1).max(axis=1)


def record(label: str, level: str, rel, rel_terms=None, kappa=None, n_flag_mismatch: int = 0,
           max_flag_window: float = 0.0, n_faces: int | None = None, bar_used=None, cap=None) -> dict:
    rel = np.atleast_1d(np.asarray(rel, dtype=np.float64))
    r = {"test": _test_id(), "label": label, "level": level, "rel_max": float(rel.max()),
         "rel": [float(x) for x in rel],
         "rel_terms_max": None if rel_terms is None else float(np.max(rel_terms)),
         "kappa_max": None if kappa is None else float(np.max(kappa)),
         "fallback": level != "strict", "n_flag_mismatch": int(n_flag_mismatch),
         "max_flag_window": float(max_flag_window), "n_faces": n_faces,
         "bar_max": None if bar_used is None else float(np.max(bar_used)), "cap": cap}
    RECORDS.append(r)
    return r


def bar(err, scale, rtol: float, kappa_fn, label: str, terms=None, n_flag_mismatch: int = 0,
        max_flag_window: float = 0.0, n_faces: int | None = None, strict: bool = False,
        cap: float | None = KAPPA_CAP):
    """err: max |gpu - oracle| per variable; scale: max |oracle| per variable;
    terms: T_v per variable (term_scale) or None; kappa_fn(): the oracle's
    one-ulp sensitivity per variable relative to `scale`.  Levels as in the
    module docstring; `strict` allows level 1 only, cap=None leaves the
    kappa bar uncapped (derivative checks, whose conditioning is recorded).
    Records the outcome and returns the record."""
    err = np.atleast_1d(np.asarray(err, dtype=np.float64))
    scale = np.atleast_1d(np.asarray(scale, dtype=np.float64))
    scale = np.where(scale > 0.0, scale, max(float(scale.max()), 1e-300))
    rel = err / scale
    rel_t = None if terms is None else err / np.maximum(np.atleast_1d(terms), 1e-300)
    if np.all(rel <= rtol):
        return record(label, "strict", rel, rel_t, None, n_flag_mismatch, max_flag_window, n_faces,
                      np.full_like(rel, rtol), cap)
    assert not strict, f"{label}: strict bar {rtol:g} missed, rel = {rel}"
    if rel_t is not None and np.all(rel_t <= rtol):
        return record(label, "terms", rel, rel_t, None, n_flag_mismatch, max_flag_window, n_faces,
                      rtol * np.atleast_1d(terms) / scale, cap)
    kappa = np.atleast_1d(np.asarray(kappa_fn(), dtype=np.float64))
    tol = np.maximum(rtol, 10.0 * kappa)
    rec = record(label, "kappa", rel, rel_t, kappa, n_flag_mismatch, max_flag_window, n_faces, tol, cap)
    over = rel > rtol
    if cap is not None:
        assert np.all(10.0 * kappa[over] <= cap), \
            f"{label}: oracle sensitivity {kappa} puts the bar above the cap {cap:g}"
    assert np.all(rel <= tol), f"{label}: rel {rel} above max(rtol, 10 kappa) = {tol}"
    return rec


def dump(path: str) -> None:
    with open(path, "w") as f:
        for r in RECORDS:
            f.write(json.dumps(r) + "\n")
