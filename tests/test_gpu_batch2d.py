"""Batched 2D problems (random cylindrical explosions and implosions in boxes
of uneven sizes, one persistent graph-replayed launch) against the
single-problem solver (bitwise: the same per-tile arithmetic and CFL steps)
and against the FP64 oracle (same status, steps and end time, L1(rho) <=
1e-10)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1908_02464_gb300 import problems as P
from tests import oracle_pool

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1908_02464_gb300 import weno  # noqa: E402


def _explosions(count, seed, n_lo=16, n_hi=64):
    params, _ = P.explosion_batch_params(count, seed=seed, n_lo=n_lo, n_hi=n_hi)
    states = [P.explosion_instance(params, i)[1] for i in range(count)]
    return params, states


def _batch(params, precision="fp64", bc_lo=(0, 0), bc_hi=(0, 0), **kw):
    h = params["h"]
    hi = np.stack([params["NX"] * h, params["NY"] * h], axis=1)
    return weno.Batch2D(params["NX"], params["NY"], (0.0, 0.0), hi, params["t_end"], precision,
                        bc_lo=bc_lo, bc_hi=bc_hi, **kw)


def _single(params, i, precision, bc_lo=(0, 0), bc_hi=(0, 0), **kw):
    prob, U = P.explosion_instance(params, i)
    prob["bc_lo"] = list(bc_lo)
    prob["bc_hi"] = list(bc_hi)
    prob.update(kw)
    s = weno.Solver(prob, precision)
    s.set_state(U)
    status = 0
    try:
        s.advance(prob["t_end"])
    except weno.WenoError as e:
        status = e.status
    V, t = s.get_state()
    k = s.time()[1]
    s.close()
    return V, t, k, status


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_batch2d_equals_single_problem_solver_bitwise(precision):
    """Sizes 5..80 per side: lines shorter than one tile, exactly one tile
    (15, 31, 63 cells) and ragged multiples."""
    params, states = _explosions(20, seed=21, n_lo=5, n_hi=80)
    b = _batch(params, precision)
    U = b.pack(states)
    b.run(U)
    st, steps, t = b.results()
    out = b.unpack(U)
    for i in range(b.count):
        V, ti, k, sti = _single(params, i, precision)
        assert st[i] == sti, i
        assert steps[i] == k and t[i] == ti, i
        assert np.array_equal(out[i], V.astype(np.float64)), i
    assert np.sum(st == 0) >= b.count - 1
    b.close()


@pytest.mark.parametrize("bcs", [((1, 2), (1, 2)), ((2, 1), (2, 0)), ((0, 1), (1, 0))])
def test_batch2d_boundaries_equal_single_solver(bcs):
    """Reflecting and periodic boundaries per direction (codes 0
    transmissive, 1 reflecting, 2 periodic), the state's waves reaching them."""
    params, states = _explosions(8, seed=22, n_lo=12, n_hi=40)
    params["t_end"] = params["t_end"] * 3.0
    b = _batch(params, "fp64", bc_lo=bcs[0], bc_hi=bcs[1])
    U = b.pack(states)
    b.run(U)
    st, steps, t = b.results()
    out = b.unpack(U)
    for i in range(b.count):
        V, ti, k, sti = _single(params, i, "fp64", bc_lo=bcs[0], bc_hi=bcs[1])
        assert st[i] == sti and steps[i] == k and t[i] == ti, i
        assert np.array_equal(out[i], V), i
    b.close()


@pytest.mark.parametrize("weights,splitting", [("is", 2), ("wang", 0), ("linear", 0)])
def test_batch2d_weights_and_splittings_equal_single_solver(weights, splitting):
    params, states = _explosions(6, seed=23)
    code = {"reg": 0, "is": 1, "wang": 2, "linear": 3}[weights]
    b = _batch(params, "fp64", weights=code, splitting=splitting)
    U = b.pack(states)
    b.run(U)
    st, steps, t = b.results()
    out = b.unpack(U)
    for i in range(b.count):
        V, ti, k, sti = _single(params, i, "fp64", weights=weights, splitting={0: "llf", 2: "rf"}[splitting])
        assert st[i] == sti and steps[i] == k and t[i] == ti, i
        assert np.array_equal(out[i], V), i
    b.close()


def test_batch2d_every_variant_and_residency_gives_the_same_states():
    params, states = _explosions(30, seed=24, n_lo=8, n_hi=70)
    b = _batch(params, "fp64")
    ref = None
    for v in range(3):
        for cap in (0, 2, 1):
            blocks = b.set_config(v, cap)
            assert 1 <= blocks <= len(states)
            U = b.pack(states)
            b.run(U)
            st, steps, t = b.results()
            if ref is None:
                ref = (U.clone(), st.copy(), steps.copy())
            else:
                assert torch.equal(U, ref[0]), (v, cap)
                assert np.array_equal(st, ref[1]) and np.array_equal(steps, ref[2]), (v, cap)
    with pytest.raises(RuntimeError):
        b.set_config(3, 0)
    b.close()


def test_batch2d_autotune_keeps_input_and_results():
    params, states = _explosions(64, seed=25)
    b = _batch(params, "fp32")
    U = b.pack(states)
    U0 = U.clone()
    choice = b.autotune(U, trial_steps=3)
    assert 0 <= choice[0] < 3 and choice[1] >= 1
    assert torch.equal(U, U0)
    b.run(U)
    ref = _batch(params, "fp32")
    U2 = ref.pack(states)
    ref.run(U2)
    assert torch.equal(U, U2)
    b.close()
    ref.close()


def test_batch2d_replay_and_nonphysical_isolation():
    params, states = _explosions(10, seed=26)
    states = [s.copy() for s in states]
    states[4][3, 2, 3] = -1.0             # negative energy
    b = _batch(params, "fp64")
    U = b.pack(states)
    b.run(U)
    A = U.clone()
    st, steps, t = b.results()
    assert st[4] == weno.WENO_ERR_NONPHYSICAL and steps[4] == 0
    assert np.array_equal(b.unpack(U)[4], states[4])
    assert np.all(np.delete(st, 4) == 0)
    U.copy_(b.pack(states))
    b.run(U)                              # graph replay on the same buffer
    assert torch.equal(U, A)
    b.close()


def test_batch2d_rejects_bad_descriptions():
    p = weno.weno_default_params()
    with pytest.raises(weno.WenoError) as e:
        weno.weno_batch2d_create([10, 2], [10, 10], (0.0, 0.0), (1.0, 1.0), [0.1, 0.1], p)
    assert e.value.status == weno.WENO_ERR_INVALID_ARG
    with pytest.raises(weno.WenoError) as e:
        weno.weno_batch2d_create([10], [10], (0.0, 0.0), (1.0, 1.0), [0.1], p, bc_lo=(2, 0), bc_hi=(0, 0))
    assert e.value.status == weno.WENO_ERR_INVALID_ARG
    p.splitting = 1
    with pytest.raises(weno.WenoError) as e:
        weno.weno_batch2d_create([10], [10], (0.0, 0.0), (1.0, 1.0), [0.1], p)
    assert e.value.status == weno.WENO_ERR_UNSUPPORTED


def test_batch2d_benchmark_batch_against_oracle():
    """The 4096-instance 2D benchmark batch in FP64: every instance that
    ends non-physical fails in the oracle as well, at the same step, and a
    sample of 256 instances spread over the size range (every 16th in size
    order) takes the oracle's steps and end time with L1(rho) <= 1e-10."""
    count, seed = 4096, 20190808
    params, _ = P.explosion_batch_params(count, seed=seed)
    states = [P.explosion_instance(params, i)[1] for i in range(count)]
    b = _batch(params, "fp64")
    U = b.pack(states)
    b.run(U)
    st, steps, t = b.results()
    out = b.unpack(U)
    b.close()
    bad = [int(i) for i in np.nonzero(st != 0)[0]]
    assert len(bad) <= count // 100
    # every non-physical instance: the oracle fails too, after the same steps
    for i, so, to, ko, _ in oracle_pool.run_many([("explosion", count, seed, i, 10 ** 9) for i in bad]):
        assert so == st[i] and ko == steps[i], (i, so, ko, steps[i])
    sample = oracle_pool.stratified(params["NX"] * params["NY"], st == 0, 256)
    l1 = oracle_pool.check_runs("explosion", count, seed, st, steps, t, [u[0] for u in out], sample, "2D batch")
    v = np.array(list(l1.values()))
    print("2D batch: %d non-physical (the oracle agrees); L1(rho) of %d sampled instances: %d above 1e-10, "
          "max %.2e, median %.2e" % (len(bad), len(sample), int(np.sum(v > 1e-10)), v.max(), np.median(v)))
