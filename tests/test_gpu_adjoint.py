"""Hand-written adjoint of the semi-discrete operator (weno_rhs_vjp) against
the oracle's dual-number Jacobian-vector product (same flags and LLF argmax:
<w, J v> = <J^T w, v> and full J^T w on small grids) and against FP64 central
differences of the GPU forward operator where no flag changes."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1908_02464_gb300 import problems as P
from tests import parity_log

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1908_02464_gb300 import weno  # noqa: E402


def _vjp(prob, U, w, precision="fp64", t=0.0):
    s = weno.Solver(prob, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    g = s.rhs_vjp(torch.from_numpy(U).to("cuda", dt), torch.from_numpy(w).to("cuda", dt), t)
    torch.cuda.synchronize()
    out = g.double().cpu().numpy()
    s.close()
    return out


def _scale(U):
    return np.abs(U).mean(axis=tuple(range(1, U.ndim)), keepdims=True)


CASES = [(1, [40], "mixed"), (1, [33], "jumps"), (2, [30, 17], "mixed"), (2, [24, 19], "smooth"),
         (3, [13, 11, 9], "mixed"), (3, [12, 9, 8], "jumps")]


@pytest.mark.parametrize("dim,n,kind", CASES)
def test_vjp_dot_product_identity_against_oracle_jvp(dim, n, kind):
    """Bar: 1e-11 relative, or ten times the oracle's own change of <w, J v>
    under one-ulp input perturbations where that is larger: the derivative of
    the weights with respect to lambda scales like tau / (lambda beta + eps)^2
    with eps = 1e-20, so on faces where lambda beta ~ eps the Jacobian itself
    is ill-conditioned.  That bar is not capped (the specification sets no
    tolerance for the derivative); every use of it is recorded with its kappa
    (tests/parity_log.py), and the full transposed Jacobians below hold to
    1e-10."""
    prob, U = P.random_state(dim, n, seed=31 + dim, kind=kind)
    rng = np.random.default_rng(7)
    prng = np.random.default_rng(99)
    w = rng.normal(size=U.shape)
    g = _vjp(prob, U, w)
    for _ in range(3):
        v = rng.normal(size=U.shape) * _scale(U)
        _, jv = orc.rhs_jvp(prob, U, v)
        lhs, rhs = np.sum(w * jv), np.sum(g * v)
        ref = np.sum(np.abs(w * jv))

        def kappa():
            k = 0.0
            for _ in range(3):
                Up = U * (1.0 + 2.220446049250313e-16 * prng.choice([-1.0, 0.0, 1.0], size=U.shape))
                _, jv2 = orc.rhs_jvp(prob, Up, v)
                k = max(k, abs(np.sum(w * jv2) - lhs))
            return k / ref

        parity_log.bar(abs(lhs - rhs), ref, 1e-11, kappa, f"<w, J v> {dim}D {kind}", cap=None)


@pytest.mark.parametrize("dim,n,bcs", [(1, [16], (0, 0)), (1, [16], (1, 1)), (2, [9, 7], (2, 2)),
                                      (2, [9, 8], (0, 1))])
def test_vjp_equals_full_transposed_jacobian(dim, n, bcs):
    """Every column of J from the oracle's JVP with unit tangents."""
    prob, U = P.random_state(dim, n, seed=4, kind="mixed")
    prob["bc_lo"] = [bcs[0]] * dim
    prob["bc_hi"] = [bcs[1]] * dim
    rng = np.random.default_rng(3)
    w = rng.normal(size=U.shape)
    g = _vjp(prob, U, w)
    ref = np.zeros(U.size)
    for k in range(U.size):
        e = np.zeros(U.size)
        e[k] = 1.0
        _, jv = orc.rhs_jvp(prob, U, e.reshape(U.shape))
        ref[k] = np.sum(w * jv)
    assert np.allclose(g.reshape(-1), ref, rtol=1e-10, atol=1e-11 * np.max(np.abs(ref)))


def test_vjp_double_mach_boundaries():
    """Inflow, DMR bottom (inflow / wall) and top (moving shock) ghosts."""
    prob, U = P.double_mach(40, 12)
    rng = np.random.default_rng(5)
    w = rng.normal(size=U.shape)
    g = _vjp(prob, U, w, t=0.01)
    for _ in range(2):
        v = rng.normal(size=U.shape) * _scale(U)
        _, jv = orc.rhs_jvp(prob, U, v, 0.01)
        assert abs(np.sum(w * jv) - np.sum(g * v)) <= 1e-11 * np.sum(np.abs(w * jv))


def test_vjp_against_central_differences_vortex_32():
    """3D periodic vortex on a 32^3 grid: FP64 central differences of the GPU
    forward operator along random directions (flags unchanged under +-h)."""
    prob, U = P.vortex3d(32)
    s = weno.Solver(prob, "fp64")
    rng = np.random.default_rng(11)
    w = rng.normal(size=U.shape)
    Ud = torch.from_numpy(U).cuda()
    g = s.rhs_vjp(Ud, torch.from_numpy(w).cuda()).cpu().numpy()
    f0 = s.face_flags(Ud).cpu().numpy()
    checked = 0
    for _ in range(4):
        v = rng.normal(size=U.shape) * _scale(U)
        h = 1e-6
        Up = torch.from_numpy(U + h * v).cuda()
        Um = torch.from_numpy(U - h * v).cuda()
        if not (np.array_equal(s.face_flags(Up).cpu().numpy(), f0) and
                np.array_equal(s.face_flags(Um).cpu().numpy(), f0)):
            continue
        fd = np.sum(w * (s.rhs(Up).cpu().numpy() - s.rhs(Um).cpu().numpy())) / (2 * h)
        assert abs(fd - np.sum(g * v)) <= 1e-6 * np.sum(np.abs(w * v)) * 1e2, (fd, np.sum(g * v))
        checked += 1
    assert checked >= 2
    s.close()


def test_autograd_function_matches_vjp():
    prob, U = P.random_state(2, [20, 16], seed=2, kind="mixed")
    s = weno.Solver(prob, "fp64")
    Ut = torch.from_numpy(U).cuda().requires_grad_(True)
    rng = np.random.default_rng(1)
    w = torch.from_numpy(rng.normal(size=U.shape)).cuda()
    r = weno.rhs_autograd(s, Ut)
    (r * w).sum().backward()
    g = s.rhs_vjp(Ut.detach(), w)
    assert torch.equal(Ut.grad, g)
    assert torch.equal(r.detach(), s.rhs(Ut.detach()))
    s.close()


def test_vjp_reads_and_writes_the_callers_arrays():
    """weno_rhs_vjp works on the caller's interior-only arrays: repeated calls
    agree bitwise whatever the output held, and an output that is one of the
    inputs is rejected."""
    prob, U = P.random_state(3, [13, 11, 9], seed=12, kind="mixed")
    s = weno.Solver(prob, "fp64")
    Ud = torch.from_numpy(U).cuda()
    w = torch.from_numpy(np.random.default_rng(4).normal(size=U.shape)).cuda()
    a = torch.full_like(Ud, float("nan"))
    b = torch.full_like(Ud, 3.0)
    s.rhs_vjp(Ud, w, 0.0, out=a)
    s.rhs_vjp(Ud, w, 0.0, out=b)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and bool(torch.isfinite(a).all())
    for out in (Ud, w):
        with pytest.raises(weno.WenoError) as e:
            weno.weno_rhs_vjp(s.ctx, Ud, w, out, 0.0)
        assert e.value.status == weno.WENO_ERR_INVALID_ARG
    s.close()


def test_fp32_vjp_close_to_fp64():
    prob, U = P.random_state(3, [16, 12, 10], seed=6, kind="smooth")
    rng = np.random.default_rng(2)
    w = rng.normal(size=U.shape)
    g64 = _vjp(prob, U, w, "fp64")
    g32 = _vjp(prob, U, w, "fp32")
    rel = np.max(np.abs(g32 - g64)) / np.max(np.abs(g64))
    assert rel < 1e-3, rel


def _weno_face_fraction(prob, U):
    s = weno.Solver(prob, "fp64")
    f = s.face_flags(torch.from_numpy(U).cuda()).cpu().numpy()
    s.close()
    return 1.0 - float(np.mean(f))


def test_vjp_entries_across_tiles():
    """A 150 x 130 grid: several adjoint tiles per line (59 cells each in
    FP64), with WENO faces in some tiles and none in others, so that the
    linear-upwind pass and the WENO pass (flagged tiles only) both write the
    gradient.  (J^T w)_k = <w, J e_k> from the oracle's JVP, at cells on both
    sides of every tile edge along x and y, and at random cells.  Bar: 1e-10
    relative, or ten times the oracle's own change of the entry under
    one-ulp input perturbations (the WENO weights' derivatives are
    ill-conditioned where lambda beta ~ eps), capped at 1e-7."""
    prob, U = P.random_state(2, [150, 130], seed=21, kind="mixed")
    frac = _weno_face_fraction(prob, U)
    assert 0.01 < frac < 0.5, frac
    rng = np.random.default_rng(8)
    prng = np.random.default_rng(99)
    w = rng.normal(size=U.shape)
    g = _vjp(prob, U, w)
    edge = [0, 1, 2, 56, 57, 58, 59, 60, 61, 62, 115, 116, 117, 118, 119, 120, 121, 127, 128, 129]
    cells = [(int(rng.integers(0, 130)), i) for i in edge + [147, 148, 149]]
    cells += [(j, int(rng.integers(0, 150))) for j in edge]
    cells += [(int(rng.integers(0, 130)), int(rng.integers(0, 150))) for _ in range(10)]
    scale = np.max(np.abs(g))
    for (j, i) in cells:
        for v in range(U.shape[0]):
            e = np.zeros_like(U)
            e[v, j, i] = 1.0
            _, jv = orc.rhs_jvp(prob, U, e)
            ref = float(np.sum(w * jv))
            den = max(abs(ref), 1e-3 * scale)

            def kappa():
                k = 0.0
                for _ in range(3):
                    Up = U * (1.0 + 2.220446049250313e-16 * prng.choice([-1.0, 0.0, 1.0], size=U.shape))
                    _, jv2 = orc.rhs_jvp(prob, Up, e)
                    k = max(k, abs(float(np.sum(w * jv2)) - ref))
                return k / den

            err = abs(g[v, j, i] - ref)
            if err > 1e-10 * den:
                parity_log.bar(err, den, 1e-10, kappa, f"(J^T w) entry {v},{j},{i} 2D mixed", cap=1e-7)


def test_vjp_hybrid_off_full_transposed_jacobian():
    """With the hybrid switch off every face takes the WENO flux: the
    linear-upwind pass takes no face and flags every tile."""
    prob, U = P.random_state(2, [9, 8], seed=5, kind="mixed")
    prob["hybrid"] = 0
    rng = np.random.default_rng(6)
    w = rng.normal(size=U.shape)
    g = _vjp(prob, U, w)
    ref = np.zeros(U.size)
    for k in range(U.size):
        e = np.zeros(U.size)
        e[k] = 1.0
        _, jv = orc.rhs_jvp(prob, U, e.reshape(U.shape))
        ref[k] = np.sum(w * jv)
    assert np.allclose(g.reshape(-1), ref, rtol=1e-10, atol=1e-11 * np.max(np.abs(ref)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kind,hybrid", [("mixed", 1), ("smooth", 0), ("jumps", 1)])
def test_vjp_tiling_on_a_replicated_state(precision, kind, hybrid):
    """A periodic 30 x 26 state and cotangent repeated 5 x 5 times on a
    150 x 130 periodic grid with the same spacing: the gradient repeats too.
    The large grid has several tiles per line (59 cells along x; along y 59
    cells in FP64 and 8 x-adjacent lines of 27 cells in FP32, ragged at the
    end), the small one a single tile per line, and the two passes split the
    faces the same way on both.  A cell at least 3 cells from the small
    grid's edges receives the same face contributions in the same order on
    both grids, so it agrees bitwise; the other cells receive their
    periodic-ghost contributions in another order and agree to rounding."""
    prob, U = P.random_state(2, [30, 26], seed=17, kind=kind)
    prob["hybrid"] = hybrid
    big = dict(prob, n=[150, 130], hi=[5.0, 5.0])
    rng = np.random.default_rng(12)
    w = rng.normal(size=U.shape)
    g_small = _vjp(prob, U, w, precision)
    g_big = _vjp(big, np.tile(U, (1, 5, 5)), np.tile(w, (1, 5, 5)), precision)
    rep = np.tile(g_small, (1, 5, 5))
    inner = np.zeros(g_small.shape[1:], dtype=bool)
    inner[3:-3, 3:-3] = True
    inner = np.tile(inner, (5, 5))
    assert np.array_equal(g_big[:, inner], rep[:, inner])
    tol = (1e-5 if precision == "fp32" else 1e-12) * np.max(np.abs(g_small))
    assert np.max(np.abs(g_big - rep)) <= tol
