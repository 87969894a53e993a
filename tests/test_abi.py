"""CPU-side checks of the C ABI: the shared library builds, loads and exports
every entry point declared in include/weno_is.h (no GPU calls here)."""
import os
import re
import subprocess

import pytest

from paper_1908_02464_gb300 import build as B
from paper_1908_02464_gb300 import weno

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "weno_is.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(weno_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_abi():
    names = _declared()
    for n in ["weno_create", "weno_destroy", "weno_set_state", "weno_get_state", "weno_rhs", "weno_step",
              "weno_advance", "weno_face_flags", "weno_conserved_totals", "weno_last_error"]:
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    lib = B.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (weno_[a-z0-9_]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_the_abi():
    assert set(_declared()) <= set(weno.SIGNATURES)
    L = weno.load()
    for n in _declared():
        assert hasattr(L, n)


def test_default_params_are_the_papers():
    p = weno.weno_default_params()
    assert p.gamma == 1.4 and p.cfl == 0.5 and p.eps == 1e-20
    assert p.c_lambda == 1.0 and p.C_thr == 1.0 and p.alpha_thr == 3 and p.hybrid == 1


def test_create_rejects_invalid_grids_without_touching_the_gpu():
    """Argument validation happens before any CUDA call."""
    from paper_1908_02464_gb300 import problems as P
    prob, _ = P.sod(200)
    g = weno.make_grid(prob)
    p = weno.make_params(prob)
    bad = []
    g1 = weno.make_grid(prob); g1.dim = 4; bad.append((g1, p))
    g2 = weno.make_grid(prob); g2.n[0] = 2; bad.append((g2, p))
    g3 = weno.make_grid(prob); g3.hi[0] = g3.lo[0]; bad.append((g3, p))
    g4 = weno.make_grid(prob); g4.bc_lo[0] = 9; bad.append((g4, p))
    g5 = weno.make_grid(prob); g5.bc_lo[0] = 2; bad.append((g5, p))   # unpaired periodic
    p2 = weno.make_params(prob); p2.precision = 7; bad.append((g, p2))
    for gg, pp in bad:
        with pytest.raises(weno.WenoError) as e:
            weno.weno_create(gg, pp)
        assert e.value.status == weno.WENO_ERR_INVALID_ARG


def test_weight_and_splitting_codes_reach_the_params():
    from paper_1908_02464_gb300 import problems as P
    prob, _ = P.blast_waves(100)   # Roe splitting
    p = weno.make_params(prob)
    assert p.splitting == 2 and p.weights == 0
    prob["weights"] = "wang"
    prob["splitting"] = "lf"
    p = weno.make_params(prob)
    assert p.splitting == 1 and p.weights == 2


def test_create_rejects_unknown_weight_rule():
    from paper_1908_02464_gb300 import problems as P
    prob, _ = P.sod(100)
    p = weno.make_params(prob)
    p.weights = 7
    with pytest.raises(weno.WenoError) as e:
        weno.weno_create(weno.make_grid(prob), p)
    assert e.value.status == weno.WENO_ERR_INVALID_ARG
