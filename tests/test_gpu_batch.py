"""Batched 1D Riemann problems (persistent, graph-replayed launch) against the
single-problem solver (bitwise: same per-face arithmetic and time steps) and
against the FP64 oracle (same step count, L1(rho) <= 1e-10)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1908_02464_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1908_02464_gb300 import weno  # noqa: E402


def _small_batch(count=24, seed=11, n_lo=60, n_hi=400):
    params, _ = P.riemann_batch_params(count, seed=seed, n_lo=n_lo, n_hi=n_hi)
    states = [P.riemann_instance(params, i)[1] for i in range(count)]
    return params, states


def _single(params, i, precision):
    """Single-problem solver; the status is WENO_ERR_NONPHYSICAL when the
    scheme produced an inadmissible state (strong contacts of cold dense and
    hot light gas can), the state then being the last admissible one."""
    prob, U = P.riemann_instance(params, i)
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
def test_batch_equals_single_problem_solver_bitwise(precision):
    params, states = _small_batch()
    b = weno.Batch(params["N"], 0.0, 1.0, params["t_end"], precision)
    U = b.pack(states)
    b.run(U)
    st, steps, t = b.results()
    out = b.unpack(U)
    ok = 0
    for i in range(b.count):
        V, ti, k, sti = _single(params, i, precision)
        assert st[i] == sti, i
        assert steps[i] == k and t[i] == ti, i
        assert np.array_equal(out[i], V.astype(np.float64)), i
        ok += st[i] == 0
    assert ok >= b.count - 2
    b.close()


@pytest.mark.parametrize("weights,splitting", [("reg", 2), ("is", 0), ("wang", 2)])
def test_batch_variants_equal_single_solver(weights, splitting):
    params, states = _small_batch(count=10, seed=13)
    code = {"reg": 0, "is": 1, "wang": 2}[weights]
    b = weno.Batch(params["N"], 0.0, 1.0, params["t_end"], "fp64", weights=code, splitting=splitting)
    U = b.pack(states)
    b.run(U)
    st, steps, t = b.results()
    out = b.unpack(U)
    for i in range(b.count):
        prob, Ui = P.riemann_instance(params, i)
        prob["weights"] = weights
        prob["splitting"] = {0: "llf", 2: "rf"}[splitting]
        s = weno.Solver(prob, "fp64")
        s.set_state(Ui)
        sti = 0
        try:
            s.advance(prob["t_end"])
        except weno.WenoError as e:
            sti = e.status
        V, ti = s.get_state()
        assert st[i] == sti and t[i] == ti and steps[i] == s.time()[1]
        assert np.array_equal(out[i], V)
        s.close()
    b.close()


def test_batch_matches_oracle():
    params, states = _small_batch(count=6, seed=5)
    b = weno.Batch(params["N"], 0.0, 1.0, params["t_end"], "fp64")
    U = b.pack(states)
    b.run(U)
    st, steps, t = b.results()
    out = b.unpack(U)
    for i in range(b.count):
        prob, Uo = P.riemann_instance(params, i)
        so, to, ko = orc.advance(prob, Uo, 0.0, prob["t_end"])
        assert so == st[i]
        assert steps[i] == ko and t[i] == to
        assert np.mean(np.abs(out[i][0] - Uo[0])) <= 1e-10
    b.close()


def test_batch_autotune_keeps_input_and_results():
    params, states = _small_batch(count=40, seed=3)
    b = weno.Batch(params["N"], 0.0, 1.0, params["t_end"], "fp64")
    U = b.pack(states)
    U0 = U.clone()
    choice = b.autotune(U, trial_steps=3)
    assert 0 <= choice[0] < 3 and choice[1] >= 1
    assert torch.equal(U, U0)
    b.run(U)
    st, steps, t = b.results()
    ref = weno.Batch(params["N"], 0.0, 1.0, params["t_end"], "fp64")
    U2 = ref.pack(states)
    ref.run(U2)
    assert torch.equal(U, U2)
    b.close()
    ref.close()


def test_batch_set_config_every_tile_and_residency_gives_the_same_states():
    # one CTA integrates one instance, and the face fluxes and the CFL maximum
    # do not depend on how the faces are cut into tiles, so every fixed
    # configuration gives the same bits
    params, states = _small_batch(count=24, seed=5)
    b = weno.Batch(params["N"], 0.0, 1.0, params["t_end"], "fp64")
    ref = None
    for v in range(3):
        for cap in (0, 2, 1):
            blocks = b.set_config(v, cap)
            assert 1 <= blocks <= len(states)
            if cap == 1:
                assert blocks == min(len(states), torch.cuda.get_device_properties(0).multi_processor_count)
            U = b.pack(states)
            b.run(U)
            st, steps, t = b.results()
            if ref is None:
                ref = (U.clone(), st.copy(), steps.copy())
            else:
                assert torch.equal(U, ref[0]), (v, cap)
                assert np.array_equal(st, ref[1]) and np.array_equal(steps, ref[2]), (v, cap)
    for bad in ((3, 0), (-1, 0), (0, -1)):
        with pytest.raises(RuntimeError):
            b.set_config(*bad)
    b.close()


def test_batch_replay_and_one_call_form():
    params, states = _small_batch(count=10, seed=8)
    b = weno.Batch(params["N"], 0.0, 1.0, params["t_end"], "fp64")
    U = b.pack(states)
    b.run(U)
    A = U.clone()
    U.copy_(b.pack(states))
    b.run(U)            # graph replay on the same buffer
    assert torch.equal(U, A)
    p = weno.weno_default_params()
    U3 = b.pack(states)
    st = weno.weno_batch_solve(params["N"], 0.0, 1.0, params["t_end"], p, U3)
    assert np.all(st == 0) and torch.equal(U3, A)
    b.close()


def test_batch_nonphysical_instance_is_isolated():
    params, states = _small_batch(count=8, seed=2)
    states = [s.copy() for s in states]
    states[3][2, 10] = -1.0          # negative energy
    b = weno.Batch(params["N"], 0.0, 1.0, params["t_end"], "fp64")
    U = b.pack(states)
    b.run(U)
    st, steps, t = b.results()
    out = b.unpack(U)
    assert st[3] == weno.WENO_ERR_NONPHYSICAL and steps[3] == 0
    assert np.array_equal(out[3], states[3])
    assert np.all(np.delete(st, 3) == 0)
    b.close()


def test_batch_rejects_bad_descriptions():
    p = weno.weno_default_params()
    with pytest.raises(weno.WenoError) as e:
        weno.weno_batch_create([100, 2], 0.0, 1.0, [0.1, 0.1], p)
    assert e.value.status == weno.WENO_ERR_INVALID_ARG
    with pytest.raises(weno.WenoError) as e:
        weno.weno_batch_create([100], 0.0, 1.0, [0.1], p, bc_lo=3)
    assert e.value.status == weno.WENO_ERR_INVALID_ARG


def test_batch_weno_face_count_equals_single_solver_counts():
    """The batch counts each WENO face once per RK stage, like the
    single-problem solver: over instances that finish, the batch's count
    equals the sum of the single solver's counts."""
    params, states = _small_batch(count=12, seed=5)
    counts, ok = [], []
    for i in range(len(states)):
        prob, U = P.riemann_instance(params, i)
        s = weno.Solver(prob, "fp64")
        s.set_state(U)
        s.weno_faces(reset=True)
        try:
            s.advance(prob["t_end"])
        except weno.WenoError:
            s.close()
            continue
        counts.append(s.weno_faces())
        ok.append(i)
        s.close()
    assert len(ok) >= 8
    b = weno.Batch(params["N"][ok], 0.0, 1.0, params["t_end"][ok], "fp64")
    U = b.pack([states[i] for i in ok])
    b.weno_faces(reset=True)
    b.run(U)
    st, steps, t = b.results()
    assert np.all(st == 0)
    assert b.weno_faces() == sum(counts) and sum(counts) > 0
    b.close()
