"""CPU pins of the oracle's boundary conditions (ghost cells).

The paper defines its boundaries only through the test problems of Sec. 4:
reflecting walls (the blast waves of Sec. 4.3), the double Mach reflection of
Sec. 4.5 (post-shock inflow on the left, a wall for x > 1/6 at the bottom with
post-shock inflow ahead of it, the exact moving shock along the top) and the
Mach 2000 jet of Sec. 4.7 (inflow where y < 0.05, ambient inflow above it,
reflecting bottom, outflow right and top).  Each test below reaches the
expected ghost values or right-hand side by a route of its own:

- a reflecting wall is the mirror plane of a periodic problem of twice the
  size whose data are mirror-symmetric, so the RHS and a few RK3 steps with
  walls must equal those of the doubled periodic problem;
- the double Mach states are derived in the test from the Rankine-Hugoniot
  relations of a Mach 10 shock, and the trace of the shock along the top
  from its 60 degree angle and its normal speed;
- the jet states are the primitive data printed in Sec. 4.7.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1908_02464_gb300 import problems as P

NG = 3


def _with_walls(prob, a, lo=True, hi=True):
    q = dict(prob)
    q["bc_lo"] = list(prob["bc_lo"])
    q["bc_hi"] = list(prob["bc_hi"])
    if lo:
        q["bc_lo"][a] = P.BC_REFLECT
    if hi:
        q["bc_hi"][a] = P.BC_REFLECT
    return q


def _mirror_doubled(prob, U, a):
    """Periodic problem on [lo - (hi - lo), hi] along a, holding U on the upper
    half and its mirror image (normal momentum negated) on the lower half."""
    dim = prob["dim"]
    ax = dim - a                      # array axis of direction a (axis 0 = variable)
    M = np.flip(U, axis=ax).copy()
    M[1 + a] = -M[1 + a]
    Ue = np.concatenate([M, U], axis=ax)
    q = dict(prob)
    q["n"] = list(prob["n"]); q["lo"] = list(prob["lo"])
    q["bc_lo"] = list(prob["bc_lo"]); q["bc_hi"] = list(prob["bc_hi"])
    q["n"][a] = 2 * prob["n"][a]
    q["lo"][a] = prob["lo"][a] - (prob["hi"][a] - prob["lo"][a])
    q["bc_lo"][a] = P.BC_PERIODIC
    q["bc_hi"][a] = P.BC_PERIODIC
    return q, np.ascontiguousarray(Ue)


def _upper_half(Ue, dim, a, n):
    sl = [slice(None)] * (dim + 1)
    sl[dim - a] = slice(n, 2 * n)
    return Ue[tuple(sl)]


@pytest.mark.parametrize("dim,n,a", [(1, [40], 0), (2, [24, 20], 0), (2, [24, 20], 1),
                                     (3, [10, 9, 8], 2)])
@pytest.mark.parametrize("kind", ["mixed", "jumps"])
def test_reflecting_wall_is_the_mirror_plane_of_a_doubled_periodic_problem(dim, n, a, kind):
    """Walls at both ends of direction a equal the doubled periodic problem
    with mirror-symmetric data: the RHS and three RK3 steps agree on [lo, hi].
    A wrong mirrored cell, a missing sign flip of the normal momentum or a
    flip of the wrong component fails this."""
    prob, U = P.random_state(dim, n, seed=90 + 7 * dim + a, kind=kind)
    wall = _with_walls(prob, a)
    per, Ue = _mirror_doubled(wall, U, a)

    dU_wall = orc.rhs(wall, U)
    dU_per = _upper_half(orc.rhs(per, Ue), dim, a, n[a])
    scale = np.max(np.abs(dU_per), axis=tuple(range(1, dim + 1)), keepdims=True)
    assert np.all(np.abs(dU_wall - dU_per) <= 1e-13 * scale)

    # the first RHS is bitwise equal; later stages differ by rounding, since
    # the lower half reconstructs the mirrored fluxes in the mirrored order
    assert np.array_equal(dU_wall, dU_per)
    assert orc.cfl_dt(wall, U) == orc.cfl_dt(per, Ue)
    Uw = U.copy(); t_w = 0.0
    Up = Ue.copy(); t_p = 0.0
    for _ in range(3):
        st_w, t_w, _ = orc.step(wall, Uw, t_w, 10.0)
        st_p, t_p, _ = orc.step(per, Up, t_p, 10.0)
        assert st_w == 0 and st_p == 0 and abs(t_w - t_p) <= 1e-13 * t_w
    ref = _upper_half(Up, dim, a, n[a])
    sc = np.max(np.abs(ref), axis=tuple(range(1, dim + 1)), keepdims=True)
    assert np.all(np.abs(Uw - ref) <= 1e-13 * sc)


@pytest.mark.parametrize("dim,n", [(1, [48]), (2, [20, 16])])
def test_reflecting_box_conserves_mass_and_energy(dim, n):
    """A closed box: no mass or energy crosses a wall (the normal velocity of
    the mirrored data is odd about the wall, so the mass and energy fluxes of
    the symmetric reconstruction vanish there), while momentum changes by the
    wall pressure."""
    prob, U = P.random_state(dim, n, seed=31 + dim, kind="mixed")
    box = prob
    for a in range(dim):
        box = _with_walls(box, a)
    dU = orc.rhs(box, U)
    tot = dU.reshape(dim + 2, -1).sum(axis=1)
    scale = np.abs(dU).reshape(dim + 2, -1).sum(axis=1)
    assert abs(tot[0]) <= 1e-13 * scale[0]
    assert abs(tot[-1]) <= 1e-13 * scale[-1]
    # momentum is not conserved: the walls push on the gas
    assert np.max(np.abs(tot[1:1 + dim]) / scale[1:1 + dim]) > 1e-6


# ---------------------------------------------------------------------------
# double Mach reflection (Sec. 4.5)
# ---------------------------------------------------------------------------

def _normal_shock_post_state(gamma, rho1, p1, mach):
    """Post-shock (rho2, un2, p2) behind a normal shock moving at Mach `mach`
    into gas at rest (Rankine-Hugoniot), and the shock speed."""
    c1 = math.sqrt(gamma * p1 / rho1)
    s = mach * c1
    rho2 = rho1 * (gamma + 1) * mach ** 2 / ((gamma - 1) * mach ** 2 + 2)
    p2 = p1 * (1 + 2 * gamma / (gamma + 1) * (mach ** 2 - 1))
    un2 = s * (1 - rho1 / rho2)              # mass flux rho1 s = rho2 (s - un2)
    return rho2, un2, p2, s


def _dmr_states():
    gamma = 1.4
    rho2, un2, p2, s = _normal_shock_post_state(gamma, 1.4, 1.0, 10.0)
    theta = math.radians(60.0)               # shock angle to the x axis
    nrm = (math.sin(theta), -math.cos(theta))  # propagation direction
    post = np.array([rho2, un2 * nrm[0], un2 * nrm[1], p2])
    pre = np.array([1.4, 0.0, 0.0, 1.0])
    # the shock line y = tan(theta) (x - x0(t)) passes x0(0) = 1/6 at y = 0 and
    # moves along x at s / sin(theta); at y = 1 it sits at x0(t) + 1 / tan(theta)
    def x_top(t):
        return 1.0 / 6.0 + s * t / math.sin(theta) + 1.0 / math.tan(theta)
    return gamma, post, pre, x_top


def _cons(gamma, w):
    rho, u, v, p = w
    return np.array([rho, rho * u, rho * v, p / (gamma - 1) + 0.5 * rho * (u * u + v * v)])


def _dmr_grid(nx=64, ny=16, seed=5):
    prob, U = P.double_mach(nx, ny)
    # a random interior, so that every ghost value below is seen to come from
    # the boundary rule and not from the initial data
    rng = np.random.Generator(np.random.Philox(seed))
    rho = rng.uniform(0.5, 2.0, size=U.shape[1:])
    u = rng.uniform(-1.0, 1.0, size=U.shape[1:])
    v = rng.uniform(-1.0, 1.0, size=U.shape[1:])
    p = rng.uniform(0.5, 3.0, size=U.shape[1:])
    return prob, P.prim_to_cons(1.4, rho, [u, v], p)


def test_double_mach_boundary_states_are_the_mach10_shock():
    gamma, post, pre, _ = _dmr_states()
    prob, _ = P.double_mach(16, 4)
    assert np.allclose(prob["bc_state"][0][:4], _cons(gamma, post), rtol=1e-14, atol=1e-14)
    assert np.allclose(prob["bc_state"][1][:4], _cons(gamma, pre), rtol=1e-14, atol=1e-14)
    assert post[0] == pytest.approx(8.0, rel=1e-14)
    assert post[3] == pytest.approx(116.5, rel=1e-14)


@pytest.mark.parametrize("t", [0.0, 0.0137, 0.05, 0.2])
def test_double_mach_top_ghosts_follow_the_moving_shock(t):
    gamma, post, pre, x_top = _dmr_states()
    prob, U = _dmr_grid()
    nx, ny = prob["n"]
    Ug = orc.fill_ghosts(prob, U, t)
    x = P.centers(0.0, 4.0, nx)
    xs = x_top(t)
    assert np.min(np.abs(x - xs)) > 1e-6      # no cell centre on the trace
    n_post = 0
    for gl in range(1, NG + 1):
        row = Ug[:, NG + ny - 1 + gl, NG:NG + nx]
        for i in range(nx):
            want = _cons(gamma, post if x[i] < xs else pre)
            n_post += x[i] < xs
            assert np.allclose(row[:, i], want, rtol=1e-13, atol=1e-13), (gl, i, x[i], xs)
    assert 0 < n_post < NG * nx


def test_double_mach_bottom_is_inflow_ahead_of_the_wedge_and_a_wall_behind():
    gamma, post, _, _ = _dmr_states()
    prob, U = _dmr_grid(seed=6)
    nx, ny = prob["n"]
    Ug = orc.fill_ghosts(prob, U, 0.03)
    x = P.centers(0.0, 4.0, nx)
    assert np.any(x < 1.0 / 6.0) and np.any(x > 1.0 / 6.0)
    for gl in range(1, NG + 1):
        row = Ug[:, NG - gl, NG:NG + nx]
        mirror = U[:, gl - 1, :].copy()          # the wall sits at y = 0
        mirror[2] = -mirror[2]
        for i in range(nx):
            want = _cons(gamma, post) if x[i] < 1.0 / 6.0 else mirror[:, i]
            assert np.allclose(row[:, i], want, rtol=1e-14, atol=1e-14), (gl, i)


def test_double_mach_left_inflow_and_right_outflow():
    gamma, post, _, _ = _dmr_states()
    prob, U = _dmr_grid(seed=7)
    nx, ny = prob["n"]
    Ug = orc.fill_ghosts(prob, U, 0.1)
    for gl in range(1, NG + 1):
        left = Ug[:, NG:NG + ny, NG - gl]
        right = Ug[:, NG:NG + ny, NG + nx - 1 + gl]
        assert np.allclose(left, _cons(gamma, post)[:, None], rtol=1e-14, atol=1e-14)
        assert np.array_equal(right, U[:, :, nx - 1])


def test_double_mach_rhs_sees_the_shock_trace_move():
    """The top boundary changes the RHS only next to the top row, and only
    between the two trace positions of the two times."""
    _, _, _, x_top = _dmr_states()
    prob, U = P.double_mach(128, 32)
    t0, t1 = 0.0, 0.01
    d0 = orc.rhs(prob, U, t0)
    d1 = orc.rhs(prob, U, t1)
    diff = np.max(np.abs(d1 - d0), axis=0)          # [ny, nx]
    rows, cols = np.nonzero(diff)
    assert rows.size > 0
    assert rows.min() >= 32 - NG                     # only the top three rows
    x = P.centers(0.0, 4.0, 128)
    dx = 4.0 / 128
    assert x[cols].min() > x_top(t0) - 4 * dx
    assert x[cols].max() < x_top(t1) + 4 * dx


# ---------------------------------------------------------------------------
# Mach 2000 jet (Sec. 4.7)
# ---------------------------------------------------------------------------

def test_jet_boundaries():
    gamma = 5.0 / 3.0
    jet = _cons(gamma, (5.0, 800.0, 0.0, 0.4127))
    amb = _cons(gamma, (0.5, 0.0, 0.0, 0.4127))
    prob, U0 = P.mach2000_jet(40, 20)
    nx, ny = prob["n"]
    rng = np.random.Generator(np.random.Philox(8))
    U = P.prim_to_cons(gamma, rng.uniform(0.5, 2.0, size=(ny, nx)),
                       [rng.uniform(-1, 1, size=(ny, nx)), rng.uniform(-1, 1, size=(ny, nx))],
                       rng.uniform(0.5, 2.0, size=(ny, nx)))
    Ug = orc.fill_ghosts(prob, U, 0.0)
    y = P.centers(0.0, 0.25, ny)
    assert np.any(y < 0.05) and np.any(y > 0.05)
    for gl in range(1, NG + 1):
        left = Ug[:, NG:NG + ny, NG - gl]
        for j in range(ny):
            want = jet if y[j] < 0.05 else amb
            assert np.allclose(left[:, j], want, rtol=1e-14, atol=1e-14), (gl, j)
        bottom = Ug[:, NG - gl, NG:NG + nx]
        mirror = U[:, gl - 1, :].copy()
        mirror[2] = -mirror[2]
        assert np.array_equal(bottom, mirror)
        assert np.array_equal(Ug[:, NG:NG + ny, NG + nx - 1 + gl], U[:, :, nx - 1])
        assert np.array_equal(Ug[:, NG + ny - 1 + gl, NG:NG + nx], U[:, ny - 1, :])
