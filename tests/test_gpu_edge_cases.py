"""Edge cases and full-size checks of the CUDA path: degenerate states,
symmetry, dimension consistency, the benchmark's 4096-problem batch against
the oracle on sampled instances, and a large 3D grid at sampled cells."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1908_02464_gb300 import problems as P
from tests import oracle_pool, parity_log

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


def test_full_benchmark_batch_against_oracle():
    """The 4096-problem batch of the benchmark (N ~ U[100, 4000]) in FP64.
    Every instance that stops non-physical stops in the oracle too, after
    the same number of completed steps (the oracle run is capped one step
    later).  A sample of 256 instances spread over the size range takes the
    oracle's steps and end time with L1(rho) <= 1e-10 (or the recorded
    conditioning bar, see tests/oracle_pool.py)."""
    count, seed = 4096, 20190807
    params, _ = P.riemann_batch_params(count, seed=seed)
    states = [P.riemann_instance(params, i)[1] for i in range(count)]
    b = weno.Batch(params["N"], 0.0, 1.0, params["t_end"], "fp64")
    U = b.pack(states)
    b.run(U)
    st, steps, t = b.results()
    out = b.unpack(U)
    b.close()
    bad = [int(i) for i in np.nonzero(st != 0)[0]]
    assert len(bad) <= count // 20
    jobs = [("riemann", count, seed, i, int(steps[i]) + 1) for i in bad]
    for i, so, to, ko, _ in oracle_pool.run_many(jobs):
        assert so == st[i] and ko == steps[i], (i, so, ko, steps[i])
    sample = oracle_pool.stratified(params["N"], st == 0, 256)
    l1 = oracle_pool.check_runs("riemann", count, seed, st, steps, t, [u[0] for u in out], sample, "1D batch")
    v = np.array(list(l1.values()))
    print("1D batch: %d non-physical (the oracle agrees); L1(rho) of %d sampled instances: %d above 1e-10, "
          "max %.2e, median %.2e" % (len(bad), len(sample), int(np.sum(v > 1e-10)), v.max(), np.median(v)))


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
    scale = np.max(np.abs(r).reshape(5, -1), axis=1)
    err = np.max(np.abs(got - ref), axis=0)

    def kappa():
        prng = np.random.default_rng(9)
        k = np.zeros(5)
        for _ in range(3):
            k = np.maximum(k, np.max(np.abs(_oracle_rhs_at(prob, U, cells, prng) - ref), axis=0))
        return k / scale

    parity_log.bar(err, scale, 1e-12, kappa, "vortex 384^3, 27 sampled cells", terms=parity_log.term_scale(prob, U))


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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["sod", "dmr", "vortex"])
def test_host_state_transfer_paths_agree(precision, case):
    """weno_set_state / weno_get_state with pageable host memory (numpy; a
    copy through a device buffer), page-locked host memory (torch pinned; the
    layout kernel reads and writes it directly) and device memory give the
    same states bitwise, and so do the steps that follow."""
    if case == "sod":
        prob, U = P.sod(300)
    elif case == "dmr":
        prob, U = P.double_mach(130, 40)
    else:
        prob, U = P.vortex3d(20)
    np_dtype = np.float64 if precision == "fp64" else np.float32
    tdtype = torch.float64 if precision == "fp64" else torch.float32
    U = U.astype(np_dtype)
    sources = {"pageable": U, "pinned": torch.from_numpy(U).pin_memory(), "device": torch.from_numpy(U).cuda()}
    outs = {}
    for name, src in sources.items():
        s = weno.Solver(prob, precision)
        s.set_state(src, 0.0)
        back = {"pageable": np.empty_like(U), "pinned": torch.empty(U.shape, dtype=tdtype).pin_memory(),
                "device": torch.empty(U.shape, dtype=tdtype, device="cuda")}
        for kind, dst in back.items():
            t = weno.weno_get_state(s.ctx, dst)
            got = dst if isinstance(dst, np.ndarray) else dst.cpu().numpy()
            assert t == 0.0 and np.array_equal(got, U), (name, kind)
        s.advance(1.0, max_steps=3)
        V = torch.empty(U.shape, dtype=tdtype).pin_memory()
        weno.weno_get_state(s.ctx, V)
        W, _ = s.get_state()
        assert np.array_equal(V.numpy(), W)
        outs[name] = W
        s.close()
    assert np.array_equal(outs["pageable"], outs["pinned"]) and np.array_equal(outs["pageable"], outs["device"])
