"""Edge cases and full-size checks of the CUDA path: degenerate states,
symmetry, dimension consistency, the benchmark's 4096-problem batch against
the oracle on sampled instances, and a large 3D grid at sampled cells."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1908_02464_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1908_02464_gb300 import weno  # noqa: E402


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n", [(1, [37]), (2, [40, 9]), (3, [11, 9, 7])])
def test_constant_state_gives_zero_rhs(precision, dim, n):
    prob, _ = P.random_state(dim, n, seed=1)
    U = np.zeros((dim + 2,) + tuple(reversed(n)))
    base = [1.3] + [0.7, -0.4, 0.2][:dim] + [4.0]
    for v in range(dim + 2):
        U[v] = base[v]
    s = weno.Solver(prob, precision)
    r = s.rhs(torch.from_numpy(U).cuda()).double().cpu().numpy()
    f = s.face_flags(torch.from_numpy(U).cuda()).cpu().numpy()
    s.close()
    tol = 1e-12 if precision == "fp64" else 2e-3
    assert np.max(np.abs(r)) <= tol * max(1.0, n[0])
    assert np.all(f == 1)


def test_mirror_symmetric_run_stays_symmetric():
    n = 200
    x = P.centers(0, 1, n)
    mid = np.abs(x - 0.5) < 0.2
    U = P.prim_to_cons(1.4, np.where(mid, 1.0, 0.125), [np.zeros(n)], np.where(mid, 1.0, 0.1))
    prob, _ = P.sod(n)
    prob["t_end"] = 0.1
    s = weno.Solver(prob, "fp64")
    s.set_state(U)
    s.advance(0.1)
    V, _ = s.get_state()
    s.close()
    assert np.allclose(V[0], V[0][::-1], rtol=1e-12, atol=1e-13)
    assert np.allclose(V[1], -V[1][::-1], rtol=1e-12, atol=1e-13)


def test_two_dimensional_data_uniform_in_y_reproduce_one_dimension():
    """A 2D grid whose data vary only along x: every row carries the 1D
    right-hand side and the y-sweep contributes nothing."""
    prob1, U1 = P.shu_osher(256)
    ny = 9
    U2 = np.zeros((4, ny, 256))
    U2[0] = U1[0]
    U2[1] = U1[1]
    U2[3] = U1[2]
    prob2 = dict(prob1, dim=2, n=[256, ny], lo=[-5.0, 0.0], hi=[5.0, 1.0], bc_lo=[0, 2], bc_hi=[0, 2])
    s1 = weno.Solver(prob1, "fp64")
    s2 = weno.Solver(prob2, "fp64")
    r1 = s1.rhs(torch.from_numpy(U1).cuda()).cpu().numpy()
    r2 = s2.rhs(torch.from_numpy(U2).cuda()).cpu().numpy()
    s1.close()
    s2.close()
    scale = np.max(np.abs(r1), axis=1)
    for j in range(ny):
        assert np.all(np.max(np.abs(r2[[0, 1, 3], j] - r1), axis=1) <= 1e-12 * scale)
        assert np.max(np.abs(r2[2, j])) <= 1e-12 * scale[1]


def test_full_benchmark_batch_sampled_against_oracle():
    """The 4096-problem batch of the benchmark (N ~ U[100, 4000]) in FP64:
    eight instances across the size range re-run by the oracle (same steps,
    same end time, L1(rho) <= 1e-10), every instance's status reported."""
    params, _ = P.riemann_batch_params(4096, seed=20190807)
    states = [P.riemann_instance(params, i)[1] for i in range(4096)]
    b = weno.Batch(params["N"], 0.0, 1.0, params["t_end"], "fp64")
    U = b.pack(states)
    b.run(U)
    st, steps, t = b.results()
    out = b.unpack(U)
    b.close()
    assert np.sum(st == 0) >= 0.9 * 4096
    order = np.argsort(params["N"])
    ok = [i for i in order if st[i] == 0]
    picks = [ok[k] for k in np.linspace(0, len(ok) - 1, 8).astype(int)]
    for i in picks:
        prob, Uo = P.riemann_instance(params, i)
        so, to, ko = orc.advance(prob, Uo, 0.0, prob["t_end"])
        assert so == 0 and ko == steps[i] and to == t[i]
        assert np.mean(np.abs(out[i][0] - Uo[0])) <= 1e-10


def test_large_3d_grid_sampled_against_oracle():
    """A 384^3 periodic vortex (FP64, ~19 GB of device buffers): RHS at
    sampled cells computed face by face by the oracle."""
    from tests.test_gpu_parity import _oracle_rhs_at
    n = 384
    prob, U = P.vortex3d(n)
    s = weno.Solver(prob, "fp64")
    r = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    s.close()
    rng = np.random.default_rng(5)
    cells = [tuple(int(x) for x in rng.integers(0, n, size=3)) for _ in range(24)]
    cells += [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 0)]
    ref = _oracle_rhs_at(prob, U, cells)
    got = np.array([r[(slice(None),) + tuple(reversed(c))] for c in cells])
    prng = np.random.default_rng(9)
    kappa = np.zeros(5)
    for _ in range(3):
        kappa = np.maximum(kappa, np.max(np.abs(_oracle_rhs_at(prob, U, cells, prng) - ref), axis=0))
    scale = np.max(np.abs(r).reshape(5, -1), axis=1)
    assert np.all(np.max(np.abs(got - ref), axis=0) <= np.maximum(1e-12 * scale, 10.0 * kappa))


def test_switch_threshold_flags_are_nested_in_the_characteristic_length():
    """eps_h = C (dx / L)^3 (Sec. 3) falls as L grows, so on fixed data every
    face that takes the WENO flux at L still takes it at 2 L, and at least as
    many faces do; the flags at L = 1 are the oracle's."""
    prob, U0 = P.shu_osher(400)
    s = weno.Solver(prob, "fp64")
    s.set_state(U0)
    s.advance(prob["t_end"])          # the developed shock / entropy-wave field
    U, _ = s.get_state()
    s.close()
    U = np.ascontiguousarray(U, dtype=np.float64)
    Ud = torch.from_numpy(U).cuda()
    prev = None
    counts = []
    for L in (0.25, 0.5, 1.0, 2.0, 4.0, 8.0):
        pr = dict(prob)
        pr["L_char"] = L
        s = weno.Solver(pr, "fp64")
        flags = s.face_flags(Ud).cpu().numpy()
        s.close()
        weno_faces = flags == 0
        if prev is not None:
            assert np.all(weno_faces[prev]), L
        prev = weno_faces
        counts.append(int(weno_faces.sum()))
        if L == 1.0:
            _, oflags, ratio = orc.rhs(prob, U, 0.0, want_flags=True)
            mism = np.nonzero(flags != oflags)[0]
            assert np.all(np.abs(ratio[mism] - 1.0) < 1e-9), len(mism)
    assert counts[-1] > counts[0], counts
