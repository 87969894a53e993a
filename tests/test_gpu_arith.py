"""Error bounds of the refined reciprocal and reciprocal square root that the
FP64 sweeps use in place of the correctly rounded division and CUDA's rsqrt
(Roe average, sound speeds, weight denominator): checked in ulps against the
exact values computed in extended precision on the host, next to CUDA's own
1.0 / x and rsqrt(x) on the same inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1908_02464_gb300 import weno

pytestmark = pytest.mark.gpu


def _inputs():
    rng = np.random.default_rng(20191908)
    # the sweeps' arguments: densities, squared sound speeds, sums of square
    # roots of densities and weight denominators (products of four terms >=
    # eps = 1e-20), over many decades
    x = 10.0 ** rng.uniform(-90.0, 90.0, 200_000)
    # mantissa sweep across two binades (the square root's seed depends on
    # the exponent's parity) and their edges
    m = np.linspace(1.0, 4.0, 40_001)
    edges = np.array([1.0, 2.0, 4.0, 0.5, 3.0, 1e-300, 1e300, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0),
                      np.nextafter(4.0, 1.0)])
    return np.concatenate([x, m, m * 1.7e-9, m * 3.3e11, edges])


def _ulps(got, exact):
    """|got - exact| in units of the spacing of float64 at the exact value
    (a correctly rounded result is within 0.5)."""
    sp = np.spacing(np.abs(exact.astype(np.float64))).astype(np.longdouble)
    return (np.abs(got.astype(np.longdouble) - exact) / sp).astype(np.float64)


def _run():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if np.finfo(np.longdouble).eps >= np.finfo(np.float64).eps:
        pytest.skip("no extended-precision long double on this host")
    x = _inputs()
    out = weno.weno_arith_selftest(torch.from_numpy(x).cuda()).cpu().numpy()
    return x, out


def test_refined_reciprocal_error_bound():
    x, (rcp_n, rcp_cuda, _, _) = _run()
    exact = np.longdouble(1) / x.astype(np.longdouble)
    assert np.all(np.isfinite(rcp_n))
    assert _ulps(rcp_cuda, exact).max() <= 0.5 + 1e-6    # CUDA's division is correctly rounded
    e = _ulps(rcp_n, exact)
    # one third-order step from the approximate seed: rounding-limited
    assert e.max() <= 1.0, e.max()
    assert np.mean(e > 0.5) < 0.05


def test_refined_rsqrt_error_bound():
    x, (_, _, rs_n, rs_cuda) = _run()
    exact = np.longdouble(1) / np.sqrt(x.astype(np.longdouble))
    assert np.all(np.isfinite(rs_n))
    e = _ulps(rs_n, exact)
    ec = _ulps(rs_cuda, exact)
    print(f"rsqrt ulps: refined max {e.max():.3f} (> 0.5: {np.mean(e > 0.5):.4f}); CUDA max {ec.max():.3f}")
    assert e.max() <= 1.0, e.max()
    assert np.mean(e > 0.5) < 0.05


def test_refined_rsqrt_rejects_inadmissible_arguments():
    """Zero, negative and non-finite arguments give NaN, so that a state with
    p <= 0 or rho <= 0 fails the admissibility checks."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x = np.array([0.0, -1.0, -1e-300, np.inf, np.nan])
    out = weno.weno_arith_selftest(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.all(np.isnan(out[2]))


def test_selftest_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = weno.load()
    assert L.weno_arith_selftest(None, 5, None) == weno.WENO_ERR_INVALID_ARG
    assert L.weno_arith_selftest(None, 0, None) == weno.WENO_OK
