"""Error bound of the Newton-refined reciprocal that the FP64 sweeps use in
place of the correctly rounded division (Roe average, weight denominator):
checked in ulps against the exact reciprocal computed in extended precision
on the host, next to CUDA's 1.0 / x on the same inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1908_02464_gb300 import weno

pytestmark = pytest.mark.gpu


def _inputs():
    rng = np.random.default_rng(20191908)
    # the sweeps' arguments: sums of square roots of densities and weight
    # denominators (products of four terms >= eps = 1e-20), over many decades
    x = 10.0 ** rng.uniform(-90.0, 90.0, 200_000)
    # mantissa sweep across one binade and its edges
    m = np.linspace(1.0, 2.0, 20_001)
    edges = np.array([1.0, 2.0, 4.0, 0.5, 3.0, 1e-300, 1e300, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0)])
    return np.concatenate([x, m, m * 1.7e-9, edges])


def _ulps(got, exact):
    """|got - exact| in units of the spacing of float64 at the exact value
    (a correctly rounded result is within 0.5)."""
    sp = np.spacing(np.abs(exact.astype(np.float64))).astype(np.longdouble)
    return (np.abs(got.astype(np.longdouble) - exact) / sp).astype(np.float64)


def test_newton_reciprocal_error_bound():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x = _inputs()
    rcp_n, rcp_cuda = weno.weno_arith_selftest(torch.from_numpy(x).cuda()).cpu().numpy()
    if np.finfo(np.longdouble).eps >= np.finfo(np.float64).eps:
        pytest.skip("no extended-precision long double on this host")
    exact = np.longdouble(1) / x.astype(np.longdouble)
    assert np.all(np.isfinite(rcp_n))
    assert _ulps(rcp_cuda, exact).max() <= 0.5 + 1e-6    # CUDA's division is correctly rounded
    e = _ulps(rcp_n, exact)
    # two quadratic Newton steps from the approximate seed: rounding-limited
    assert e.max() <= 1.0, e.max()
    assert np.mean(e > 0.5) < 0.05


def test_selftest_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = weno.load()
    assert L.weno_arith_selftest(None, 5, None) == weno.WENO_ERR_INVALID_ARG
    assert L.weno_arith_selftest(None, 0, None) == weno.WENO_OK
