"""The allocation-free totals entry point against the context-based one.

weno_conserved_totals_noalloc serves callers that cannot allocate device
memory where they need the totals (applications whose device memory belongs
to their own pool, time-stepping loops with a fixed budget).  Its scratch is a
file-scope device array shared by all calls, so the test calls it twice in a
row, on two different states, and compares each result with
weno_conserved_totals of a context holding the same state.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_1908_02464_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1908_02464_gb300 import weno  # noqa: E402

RTOL = 1e-12


def _both(prob, U, precision):
    s = weno.Solver(prob, precision)
    s.set_state(U)
    ref = s.totals()
    V, _ = s.get_state(device=True)
    dim = prob["dim"]
    n = prob["n"][:dim]
    dx = [(prob["hi"][d] - prob["lo"][d]) / prob["n"][d] for d in range(dim)]
    out = torch.full((dim + 2,), float("nan"), dtype=torch.float64, device="cuda")
    weno.weno_conserved_totals_noalloc(dim, n, dx, precision, V, out)
    torch.cuda.synchronize()
    s.close()
    return ref, out.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_totals_match_context_totals_twice(precision):
    prob1, U1 = P.double_mach(300, 77)
    prob2, U2 = P.random_state(3, [40, 33, 17], seed=4, kind="mixed")
    prob3, U3 = P.sod(4099)          # 1D, two blocks of the partial-sum scratch
    for prob, U in ((prob1, U1), (prob2, U2), (prob3, U3)):
        ref, got = _both(prob, U, precision)
        assert np.all(np.isfinite(got))
        assert np.allclose(got, ref, rtol=RTOL, atol=1e-14 * np.max(np.abs(ref)))


def test_noalloc_totals_rejects_oversized_grids():
    big = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(weno.WenoError) as e:
        weno.weno_conserved_totals_noalloc(3, [512, 512, 257], [1.0, 1.0, 1.0], "fp64", big, out)
    assert e.value.status == weno.WENO_ERR_INVALID_ARG
    # a product of extents that would overflow a 64-bit count is rejected too
    with pytest.raises(weno.WenoError) as e:
        weno.weno_conserved_totals_noalloc(3, [2 ** 31 - 1] * 3, [1.0, 1.0, 1.0], "fp64", big, out)
    assert e.value.status == weno.WENO_ERR_INVALID_ARG
