"""The oracle and the input generators against the numbers the paper prints.

tests/golden/reconstruction_coefficients.txt holds the coefficients of
Eq. eq6, eq8, eq11, eq15, eq18 and Eq. linearupwind as printed; the oracle's
reconstruction internals are evaluated against those forms on random data.
tests/golden/problem_setups.txt holds the initial and boundary data of the
test problems of Sec. 4 as printed; the generators of problems.py are checked
against them, with the readings the fixture names where the build differs.
"""
import configparser
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1908_02464_gb300 import problems as P

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
rng = np.random.default_rng(908)


def _q(s: str) -> float:
    return float(Fraction(s))


def _coeffs():
    out = {}
    with open(os.path.join(GOLD, "reconstruction_coefficients.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, body = (x.strip() for x in line.split("|", 1))
            out[key] = body
    return out


C = _coeffs()


def _row(body):
    return np.array([_q(t) for t in body.split()])


def _squares(body):
    """[(w, a)] of sum_i w_i (a_i . f)^2"""
    terms = []
    for t in body.split(";"):
        w, a = t.split(":")
        terms.append((_q(w.strip()), np.array([_q(x) for x in a.split()])))
    return terms


def _eval_squares(body, f5):
    return sum(w * float(a @ f5) ** 2 for w, a in _squares(body))


def _eval_error(body, f5):
    fac, mono = body.split(":")
    fac = _q(fac.strip())
    if fac == 0.0:
        return 0.0
    s = 0.0
    for t in mono.split(";"):
        c, a, b = t.split()
        s += _q(c) * f5[int(a) + 2] * f5[int(b) + 2]
    return fac * s


@pytest.mark.parametrize("trial", range(10))
def test_candidate_fluxes_are_eq6(trial):
    f5 = rng.normal(size=5) * 10 ** rng.uniform(-3, 3)
    _, det = orc.recon(f5, 0.5)
    for k in range(4):
        ref = float(_row(C[f"candidate {k}"]) @ f5)
        assert det["q"][k] == pytest.approx(ref, rel=1e-13, abs=1e-14 * np.abs(f5).max())


@pytest.mark.parametrize("trial", range(10))
def test_indicators_are_eq11(trial):
    f5 = rng.normal(size=5) * 10 ** rng.uniform(-3, 3)
    _, det = orc.recon(f5, 0.5)
    scale = np.abs(f5).max() ** 2
    for k in range(4):
        ref = _eval_squares(C[f"indicator beta{k}"], f5)
        assert det["beta"][k] == pytest.approx(ref, rel=1e-12, abs=1e-14 * scale)
    assert det["tau5"] == pytest.approx(_eval_squares(C["indicator tau5"], f5), rel=1e-11, abs=1e-13 * scale)


@pytest.mark.parametrize("trial", range(10))
def test_error_terms_are_eq18(trial):
    f5 = rng.normal(size=5) * 10 ** rng.uniform(-3, 3)
    _, det = orc.recon(f5, 0.5)
    scale = np.abs(f5).max() ** 2
    for k in range(4):
        ref = _eval_error(C[f"error E{k}"], f5)
        assert det["E"][k] == pytest.approx(ref, rel=1e-11, abs=1e-13 * scale)


def test_wang_weights_use_the_beta01_of_eq15():
    """Eq. eq14: alpha_0 / d_0 - 1 = tau5^2 / ((beta_0 + eps)(beta01 + eps))."""
    d = _row(C["optimal"])
    for _ in range(10):
        f5 = rng.normal(size=5)
        _, det = orc.recon(f5, 0.0, weights="wang", eps=1e-20)
        b01 = _eval_squares(C["indicator beta01"], f5)
        tau = _eval_squares(C["indicator tau5"], f5)
        b0 = _eval_squares(C["indicator beta0"], f5)
        b1 = _eval_squares(C["indicator beta1"], f5)
        assert det["alpha"][0] == pytest.approx(d[0] * (1 + tau / (b0 + 1e-20) * tau / (b01 + 1e-20)), rel=1e-11)
        assert det["alpha"][1] == pytest.approx(d[1] * (1 + tau / (b1 + 1e-20) * tau / (b01 + 1e-20)), rel=1e-11)


def test_optimal_weights_are_eq8():
    d = _row(C["optimal"])
    assert d.sum() == pytest.approx(1.0, abs=1e-15)
    for _ in range(5):
        _, det = orc.recon(rng.normal(size=5), 0.0)
        assert np.allclose(det["omega"], d, rtol=0, atol=1e-15)


def test_linear_scheme_is_the_d_weighted_candidates():
    """The oracle's linear reconstruction on unit data reproduces
    sum_k d_k c_k from the printed Eq. eq6 and eq8."""
    d = _row(C["optimal"])
    comb = sum(d[k] * _row(C[f"candidate {k}"]) for k in range(4))
    for m in range(5):
        e = np.zeros(5)
        e[m] = 1.0
        r, _ = orc.recon(e, 0.0, weights="linear")
        assert r == pytest.approx(comb[m], abs=1e-15)
    # the printed values combine into the fifth-order upwind flux (2,-13,47,27,-3)/60
    assert np.allclose(comb * 60.0, [2, -13, 47, 27, -3], atol=1e-12)


def test_printed_upwind_central_flux_is_the_symmetric_linear_flux():
    """central6 of Eq. linearupwind = the d-weighted reconstruction of f/2
    from the left plus its mirror from the right (the printed numbers agree
    with each other)."""
    d = _row(C["optimal"])
    comb = sum(d[k] * _row(C[f"candidate {k}"]) for k in range(4))
    left = np.concatenate([comb, [0.0]])
    right = np.concatenate([[0.0], comb[::-1]])
    (w, a), = _squares(C["central6"])
    assert np.allclose(0.5 * (left + right), w * a, atol=1e-15)
    # the difference of Eq. eq28 is (left - right) / 2 of the same flux, i.e.
    # the linear-scheme dissipation acting on the split part alpha v
    (w2, a2), = _squares(C["difference6"])
    assert np.allclose(0.5 * (left - right), w2 * a2, atol=1e-15)


# ---------------------------------------------------------------- problems

S = configparser.ConfigParser()
S.read(os.path.join(GOLD, "problem_setups.txt"))


def _floats(sec, key):
    return [float(x) for x in S[sec][key].split()]


def _prim(prob, U):
    g = prob["gamma"]
    rho = U[0]
    vel = [U[1 + k] / rho for k in range(prob["dim"])]
    ke = 0.5 * rho * sum(v * v for v in vel)
    return rho, vel, (g - 1.0) * (U[-1] - ke)


@pytest.mark.parametrize("name,fn", [("sod", P.sod), ("lax", P.lax), ("p123", P.problem_123)])
def test_shock_tubes_match_sec_4_2(name, fn):
    prob, U = fn(int(S[name]["cells"]))
    rho, (u,), p = _prim(prob, U)
    L, R = _floats(name, "left"), _floats(name, "right")
    assert (rho[0], u[0], p[0]) == pytest.approx(tuple(L), rel=1e-12)
    assert (rho[-1], u[-1], p[-1]) == pytest.approx(tuple(R), rel=1e-12)
    assert prob["x0"] == float(S[name]["interface"])
    assert [prob["lo"][0], prob["hi"][0]] == _floats(name, "domain")
    t_print = float(S[name]["t_end"])
    if "reading" in S[name]:
        assert prob["t_end"] == float(S[name]["reading"].split()[1])
    else:
        assert prob["t_end"] == t_print
    assert prob["splitting"] == S["general"]["splitting_1d"]


def test_blast_waves_match_sec_4_3():
    n = int(S["blast"]["cells"])
    prob, U = P.blast_waves(n)
    rho, (u,), p = _prim(prob, U)
    x = P.centers(0.0, 1.0, n)
    a, b = _floats("blast", "interfaces")
    for sel, key in [(x < a, "left"), ((x > a) & (x < b), "middle"), (x > b, "right")]:
        st = _floats("blast", key)
        assert np.allclose(rho[sel], st[0]) and np.allclose(u[sel], st[1]) and np.allclose(p[sel], st[2])
    assert prob["t_end"] == float(S["blast"]["t_end"])
    assert prob["splitting"] == "rf"   # Roe splitting
    assert prob["bc_lo"] == [P.BC_REFLECT] and prob["bc_hi"] == [P.BC_REFLECT]


def test_shu_osher_matches_sec_4_4_under_its_reading():
    prob, U = P.shu_osher(400)
    rho, (u,), p = _prim(prob, U)
    L = _floats("shu_osher", "left")
    assert rho[0] == pytest.approx(L[0], rel=1e-12) and u[0] == pytest.approx(L[1], rel=1e-12)
    assert p[0] == pytest.approx(L[2], rel=1e-5)   # printed 10.3333, workload 10.33333
    x = P.centers(-5.0, 5.0, 400)
    right = x > -4.0
    assert np.allclose(rho[right], 1.0 + 0.2 * np.sin(5.0 * x[right]), rtol=1e-13)
    assert np.allclose(u[right], 0.0) and np.allclose(p[right], 1.0)
    # the printed interface x = 1 on [0, 10] is x = -4 on the shifted domain
    lo, hi = _floats("shu_osher", "domain")
    assert float(S["shu_osher"]["interface"]) - lo == pytest.approx(-4.0 - prob["lo"][0])
    assert hi - lo == prob["hi"][0] - prob["lo"][0]
    assert prob["t_end"] == float(S["shu_osher"]["t_end"])


def test_double_mach_matches_sec_4_5_to_printed_precision():
    prob, U = P.double_mach(64, 16)
    pre, post = _floats("double_mach", "pre"), _floats("double_mach", "post")
    assert P.DMR_PRE == pytest.approx(tuple(pre), abs=0)
    # printed to three or four digits; the build uses the exact Mach 10 values
    assert P.DMR_POST[0] == post[0]
    assert P.DMR_POST[1] == pytest.approx(post[1], abs=5e-4)
    assert P.DMR_POST[2] == pytest.approx(post[2], abs=5e-4)
    assert P.DMR_POST[3] == pytest.approx(post[3], rel=3e-3)
    assert math.sqrt(3.0) == pytest.approx(float(S["double_mach"]["shock_slope"]), abs=5e-4)
    assert 1.0 / 6.0 == pytest.approx(float(S["double_mach"]["shock_x0"]), abs=5e-5)
    assert [prob["lo"][0], prob["hi"][0], prob["lo"][1], prob["hi"][1]] == _floats("double_mach", "domain")
    assert prob["t_end"] == float(S["double_mach"]["t_end"])
    rho, (u, v), p = _prim(prob, U)
    assert rho[0, 0] == pytest.approx(post[0]) and rho[0, -1] == pytest.approx(pre[0])


def test_mach2000_jet_matches_sec_4_7():
    nx, ny = (int(x) for x in S["jet"]["cells"].split())
    prob, U = P.mach2000_jet(nx, ny)
    amb, jet = _floats("jet", "ambient"), _floats("jet", "jet")
    assert prob["gamma"] == pytest.approx(_q(S["jet"]["gamma"]))
    assert prob["cfl"] == float(S["jet"]["cfl"]) and prob["t_end"] == float(S["jet"]["t_end"])
    assert [prob["lo"][0], prob["hi"][0], prob["lo"][1], prob["hi"][1]] == _floats("jet", "domain")
    rho, (u, v), p = _prim(prob, U)
    assert np.allclose(rho, amb[0]) and np.allclose(u, 0) and np.allclose(v, 0) and np.allclose(p, amb[3])
    g = prob["gamma"]
    for k, st in enumerate((jet, amb)):
        bs = prob["bc_state"][k]
        assert bs[0] == pytest.approx(st[0])
        assert bs[1] / bs[0] == pytest.approx(st[1])
        assert (g - 1.0) * (bs[3] - 0.5 * bs[1] ** 2 / bs[0]) == pytest.approx(st[3], rel=1e-9)
    assert prob["bc_lo"] == [P.BC_JET, P.BC_REFLECT]
    assert prob["bc_hi"] == [P.BC_TRANSMISSIVE, P.BC_TRANSMISSIVE]


# ------------------------------------------ Shu-Osher high-resolution reference

def _shu_osher_ref():
    vals = [float(l) for l in open(os.path.join(GOLD, "shu_osher_rho_ref400.txt")) if not l.startswith("#")]
    return np.array(vals)


def test_shu_osher_reference_file_is_the_oracles():
    """The stored 3200-cell reference is what the committed generator computes
    with the oracle (rounding differences between compilers aside)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("mkref", os.path.join(GOLD, "make_shu_osher_reference.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    rho, _ = mk.reference()
    ref = _shu_osher_ref()
    assert ref.shape == (400,)
    assert np.max(np.abs(rho - ref)) <= 1e-9


def test_shu_osher_400_converges_toward_the_reference():
    """The 400-cell oracle run is close to the 3200-cell reference (the
    entropy waves behind the shock are the resolution-limited part), and a
    200-cell run is farther away."""
    ref = _shu_osher_ref()
    errs = {}
    for n in (200, 400):
        prob, U = P.shu_osher(n)
        U = np.ascontiguousarray(U)
        st, t, _ = orc.advance(prob, U, 0.0, prob["t_end"])
        assert st == 0
        r = ref if n == 400 else ref.reshape(200, 2).mean(axis=1)
        errs[n] = np.mean(np.abs(U[0] - r))
    assert errs[400] < 0.05 and errs[400] < 0.6 * errs[200], errs
