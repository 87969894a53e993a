"""Seeded, synthetic initial data and grids of the test problems.

This module is shared by the CUDA path and by the CPU oracle; it holds no part
of the numerical method.  Each function returns a problem description (a dict
with the grid, boundary codes, gas constants and end time) together with the
initial conservative state ``U`` of shape ``[nvar, (nz,) (ny,) nx]`` in FP64
(``nvar`` = dim + 2; the scalar advection problem has ``dim = 0``,
``nvar = 1``).  The conversion from primitive data uses the ideal-gas total
energy E = p/(gamma-1) + rho |u|^2 / 2 that defines the problems (Sec. 2.4).

Grids are cell-centred: x_i = lo + (i + 1/2) dx.

Problems follow Sec. 4 of the paper (Sod and Lax shock tubes, 123 problem,
two blast waves, Shu-Osher, double Mach reflection) and the derived
workloads: smooth periodic advection, batches of random 1D Riemann problems
and of random 2D cylindrical explosions, and a periodic 3D vortex.
"""
from __future__ import annotations

import math

import numpy as np

BC_TRANSMISSIVE, BC_REFLECT, BC_PERIODIC, BC_INFLOW, BC_DMR_BOTTOM, BC_DMR_TOP, BC_JET = range(7)


def centers(lo: float, hi: float, n: int) -> np.ndarray:
    dx = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * dx


def prim_to_cons(gamma: float, rho, vel, p) -> np.ndarray:
    """Stack (rho, rho*u_k..., E) from primitive arrays; vel is a list."""
    rho = np.asarray(rho, dtype=np.float64)
    mom = [rho * np.asarray(u, dtype=np.float64) for u in vel]
    ke = sum(0.5 * rho * np.asarray(u, dtype=np.float64) ** 2 for u in vel)
    E = np.asarray(p, dtype=np.float64) / (gamma - 1.0) + ke
    return np.stack([rho] + mom + [E]).astype(np.float64)


def _base(dim, n, lo, hi, bc_lo, bc_hi, t_end, name, **kw):
    d = dict(name=name, dim=dim, n=list(n), lo=list(lo), hi=list(hi), bc_lo=list(bc_lo),
             bc_hi=list(bc_hi), gamma=1.4, cfl=0.5, eps=1e-20, c_lambda=1.0, C_thr=1.0,
             L_char=1.0, alpha_thr=3, hybrid=1, weights="reg", splitting="llf",
             bc_state=[[0.0] * 5, [0.0] * 5], adv_speed=1.0, dt_fixed=0.0, t_end=t_end)
    d.update(kw)
    return d


def riemann_1d(n: int, WL, WR, t_end: float, lo=0.0, hi=1.0, x0=0.5, gamma=1.4, name="riemann"):
    """Shock tube: primitive states WL=(rho,u,p) for x < x0, WR otherwise."""
    x = centers(lo, hi, n)
    left = x < x0
    rho = np.where(left, WL[0], WR[0])
    u = np.where(left, WL[1], WR[1])
    p = np.where(left, WL[2], WR[2])
    prob = _base(1, [n], [lo], [hi], [BC_TRANSMISSIVE], [BC_TRANSMISSIVE], t_end, name,
                 gamma=gamma, x0=x0, WL=list(map(float, WL)), WR=list(map(float, WR)))
    return prob, prim_to_cons(gamma, rho, [u], p)


def sod(n: int = 200):
    """Sod tube of Sec. 4.2, t = 0.2."""
    return riemann_1d(n, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.2, name="sod")


def lax(n: int = 200):
    """Lax tube of Sec. 4.2, t = 0.14."""
    return riemann_1d(n, (0.445, 0.698, 3.528), (0.5, 0.0, 0.571), 0.14, name="lax")


def problem_123(n: int = 200):
    """123 problem of Sec. 4.2, t = 1 (two strong rarefactions)."""
    return riemann_1d(n, (1.0, -2.0, 0.4), (1.0, 2.0, 0.4), 1.0, name="123")


def blast_waves(n: int = 400):
    """Two interacting blast waves of Sec. 4.3, reflecting walls, t = 0.038."""
    x = centers(0.0, 1.0, n)
    p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
    prob = _base(1, [n], [0.0], [1.0], [BC_REFLECT], [BC_REFLECT], 0.038, "blast",
                 splitting="rf")
    return prob, prim_to_cons(1.4, np.ones(n), [np.zeros(n)], p)


def shu_osher(n: int = 400):
    """Shock / entropy-wave interaction on [-5, 5] (Sec. 4.4 shifted), t = 1.8."""
    x = centers(-5.0, 5.0, n)
    left = x < -4.0
    rho = np.where(left, 3.857143, 1.0 + 0.2 * np.sin(5.0 * x))
    u = np.where(left, 2.629369, 0.0)
    p = np.where(left, 10.33333, 1.0)
    prob = _base(1, [n], [-5.0], [5.0], [BC_TRANSMISSIVE], [BC_TRANSMISSIVE], 1.8, "shu_osher")
    return prob, prim_to_cons(1.4, rho, [u], p)


def advection_sine(n: int):
    """Scalar u_t + u_x = 0 on [-1, 1], periodic, u0 = sin(pi x), t = 0.5,
    dt = 0.5 dx^(5/3) so that the RK3 error does not mask fifth order."""
    x = centers(-1.0, 1.0, n)
    dx = 2.0 / n
    prob = _base(0, [n], [-1.0], [1.0], [BC_PERIODIC], [BC_PERIODIC], 0.5, "advection",
                 adv_speed=1.0, dt_fixed=0.5 * dx ** (5.0 / 3.0))
    return prob, np.sin(np.pi * x)[None, :].astype(np.float64)


def density_wave(n: int, amp: float = 0.2):
    """Euler entropy wave rho = 1 + amp sin(pi x), u = 1, p = 1 on [-1, 1],
    periodic; the exact solution is the translate rho(x - t).  t = 0.5,
    dt = 0.5 dx^(5/3)."""
    x = centers(-1.0, 1.0, n)
    dx = 2.0 / n
    prob = _base(1, [n], [-1.0], [1.0], [BC_PERIODIC], [BC_PERIODIC], 0.5, "density_wave",
                 dt_fixed=0.5 * dx ** (5.0 / 3.0), amp=amp)
    rho = 1.0 + amp * np.sin(np.pi * x)
    return prob, prim_to_cons(1.4, rho, [np.ones(n)], np.ones(n))


DMR_POST = (8.0, 8.25 * math.cos(math.pi / 6.0), -8.25 * math.sin(math.pi / 6.0), 116.5)
DMR_PRE = (1.4, 0.0, 0.0, 1.0)


def double_mach(nx: int = 2048, ny: int = 512):
    """Double Mach reflection of Sec. 4.5 on [0,4] x [0,1], t = 0.2.

    Mach-10 shock through (1/6, 0) at 60 degrees; post-shock state
    rho = 8, (u, v) = 8.25 (cos 30, -sin 30), p = 116.5.  Left: post-shock
    inflow; right: transmissive; bottom: post-shock for x < 1/6 else
    reflecting wall; top: exact moving shock."""
    gamma = 1.4
    x = centers(0.0, 4.0, nx)[None, :]
    y = centers(0.0, 1.0, ny)[:, None]
    post = y > math.sqrt(3.0) * (x - 1.0 / 6.0)
    shape = (ny, nx)
    rho = np.where(post, DMR_POST[0], DMR_PRE[0]) * np.ones(shape)
    u = np.where(post, DMR_POST[1], DMR_PRE[1]) * np.ones(shape)
    v = np.where(post, DMR_POST[2], DMR_PRE[2]) * np.ones(shape)
    p = np.where(post, DMR_POST[3], DMR_PRE[3]) * np.ones(shape)
    Upost = prim_to_cons(gamma, np.array(DMR_POST[0]), [np.array(DMR_POST[1]), np.array(DMR_POST[2])],
                         np.array(DMR_POST[3]))
    Upre = prim_to_cons(gamma, np.array(DMR_PRE[0]), [np.array(DMR_PRE[1]), np.array(DMR_PRE[2])],
                        np.array(DMR_PRE[3]))
    prob = _base(2, [nx, ny], [0.0, 0.0], [4.0, 1.0], [BC_INFLOW, BC_DMR_BOTTOM],
                 [BC_TRANSMISSIVE, BC_DMR_TOP], 0.2, "double_mach",
                 bc_state=[list(map(float, Upost)) + [0.0], list(map(float, Upre)) + [0.0]])
    return prob, prim_to_cons(gamma, rho, [u, v], p)


def mach2000_jet(nx: int = 640, ny: int = 160):
    """Mach 2000 jet of Sec. 4.7 on [0,1] x [0,0.25], gamma = 5/3, CFL 0.25,
    t = 0.001.  Ambient (rho, u, v, p) = (0.5, 0, 0, 0.4127); the left
    boundary injects (5, 800, 0, 0.4127) where y < 0.05 and the ambient state
    elsewhere; reflecting bottom, outflow right and top.

    Global Lax-Friedrichs splitting, as Sec. 4 uses for its 2D cases, and the
    regularization parameter lambda = (60 dv / rho~)^2, i.e. Eq. eq29 with
    the detector's fifth difference taken without the 1/60 of Eq. eq28
    (c_lambda = 3600 on the eq28 form).  With c = 1 on the eq28 form the
    method stops with a negative pressure within 60 steps, at odds with the
    robustness Sec. 4.7 reports; the hybrid threshold keeps the eq28 form."""
    gamma = 5.0 / 3.0
    amb = (0.5, 0.0, 0.0, 0.4127)
    jet = (5.0, 800.0, 0.0, 0.4127)
    shape = (ny, nx)

    def cons(s):
        return prim_to_cons(gamma, np.array(s[0]), [np.array(s[1]), np.array(s[2])], np.array(s[3]))
    prob = _base(2, [nx, ny], [0.0, 0.0], [1.0, 0.25], [BC_JET, BC_REFLECT], [BC_TRANSMISSIVE, BC_TRANSMISSIVE],
                 0.001, "mach2000_jet", gamma=gamma, cfl=0.25, splitting="lf", c_lambda=3600.0,
                 bc_state=[list(map(float, cons(jet))) + [0.0], list(map(float, cons(amb))) + [0.0]])
    U = prim_to_cons(gamma, np.full(shape, amb[0]), [np.zeros(shape), np.zeros(shape)], np.full(shape, amb[3]))
    return prob, U


def vortex3d(n: int = 256):
    """Periodic 3D vortex on [0, 2pi]^3: rho = 1, u = sin x cos y cos z,
    v = -cos x sin y cos z, w = 0, p = 100 + (cos 2x + cos 2y)(cos 2z + 2)/16."""
    L = 2.0 * math.pi
    x = centers(0.0, L, n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    p = 100.0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    prob = _base(3, [n, n, n], [0.0] * 3, [L] * 3, [BC_PERIODIC] * 3, [BC_PERIODIC] * 3, 1.0, "vortex3d")
    return prob, prim_to_cons(1.4, np.ones_like(u), [u, v, w], p)


def random_state(dim: int, n, seed: int, kind: str = "mixed", gamma: float = 1.4):
    """Seeded random admissible state on a periodic box [0,1]^dim.

    kind = "smooth": a few low Fourier modes; "jumps": piecewise-constant
    random slabs; "mixed": smooth background plus jumps (both face types)."""
    rng = np.random.Generator(np.random.Philox(seed))
    n = list(n)
    shape = tuple(reversed(n))
    coords = np.meshgrid(*[centers(0.0, 1.0, m) for m in reversed(n)], indexing="ij")

    def smooth_field(base, amp):
        f = np.full(shape, base)
        for _ in range(3):
            k = rng.integers(1, 4, size=dim)
            ph = rng.uniform(0, 2 * np.pi)
            arg = sum(2 * np.pi * k[a] * coords[dim - 1 - a] for a in range(dim)) + ph
            f = f + amp * rng.uniform(0.2, 1.0) * np.sin(arg)
        return f

    def jump_field(lo_, hi_):
        f = np.full(shape, rng.uniform(lo_, hi_))
        for _ in range(4):
            a = rng.integers(0, dim)
            x0, x1 = np.sort(rng.uniform(0, 1, size=2))
            m = (coords[dim - 1 - a] >= x0) & (coords[dim - 1 - a] < x1)
            f = np.where(m, rng.uniform(lo_, hi_), f)
        return f

    if kind == "smooth":
        rho = smooth_field(1.0, 0.2)
        p = smooth_field(1.0, 0.2)
        vel = [smooth_field(0.0, 0.5) for _ in range(dim)]
    elif kind == "jumps":
        rho = jump_field(0.2, 3.0)
        p = jump_field(0.2, 5.0)
        vel = [jump_field(-1.0, 1.0) for _ in range(dim)]
    else:
        rho = smooth_field(1.0, 0.2) * jump_field(0.5, 2.0)
        p = smooth_field(1.0, 0.2) * jump_field(0.5, 3.0)
        vel = [smooth_field(0.0, 0.5) + jump_field(-0.5, 0.5) for _ in range(dim)]
    prob = _base(dim, n, [0.0] * dim, [1.0] * dim, [BC_PERIODIC] * dim, [BC_PERIODIC] * dim, 1.0,
                 f"random_{kind}", gamma=gamma)
    return prob, prim_to_cons(gamma, rho, vel, p)


def riemann_batch_params(count: int = 4096, seed: int = 20190807, gamma: float = 1.4,
                         n_lo: int = 100, n_hi: int = 4000):
    """Random 1D Riemann problems on [0, 1] with the interface at 0.5.

    N ~ U{n_lo..n_hi}; rho, p log-uniform in [0.01, 10] per side; u ~ U[-2, 2].
    Draws are redrawn from the same stream when the data generate a vacuum
    (2(c_L + c_R)/(gamma - 1) <= u_R - u_L, here with a factor-two margin) or
    a star pressure below 1e-3 min(p_L, p_R).  A star pressure below
    min(p_L, p_R) means two rarefactions, for which the closed form
    p* = [(c_L + c_R - (gamma-1)(u_R - u_L)/2) / (c_L p_L^-z + c_R p_R^-z)]^(1/z),
    z = (gamma-1)/(2 gamma), is exact, so the test needs no iteration.
    t_end = 0.2 / max(|u_L| + c_L, |u_R| + c_R).
    Returns a dict of arrays (N, WL[count,3], WR[count,3], t_end) and the
    number of redraws."""
    rng = np.random.Generator(np.random.Philox(seed))
    N = np.zeros(count, dtype=np.int64)
    WL = np.zeros((count, 3)); WR = np.zeros((count, 3)); T = np.zeros(count)
    redraws = 0
    i = 0
    while i < count:
        n = int(rng.integers(n_lo, n_hi + 1))
        rl, rr, pl, pr = np.exp(rng.uniform(np.log(0.01), np.log(10.0), size=4))
        ul, ur = rng.uniform(-2.0, 2.0, size=2)
        cl = math.sqrt(gamma * pl / rl); cr = math.sqrt(gamma * pr / rr)
        if 2.0 * (cl + cr) / (gamma - 1.0) <= 2.0 * (ur - ul):
            redraws += 1
            continue
        z = (gamma - 1.0) / (2.0 * gamma)
        num = cl + cr - 0.5 * (gamma - 1.0) * (ur - ul)
        p_tr = (num / (cl * pl ** (-z) + cr * pr ** (-z))) ** (1.0 / z)
        if p_tr < 1e-3 * min(pl, pr):
            redraws += 1
            continue
        N[i] = n; WL[i] = (rl, ul, pl); WR[i] = (rr, ur, pr)
        T[i] = 0.2 / max(abs(ul) + cl, abs(ur) + cr)
        i += 1
    return dict(N=N, WL=WL, WR=WR, t_end=T, gamma=gamma), redraws


def explosion_batch_params(count: int = 4096, seed: int = 20190808, gamma: float = 1.4, n_lo: int = 16,
                           n_hi: int = 64, h: float = 1.0 / 64.0):
    """Random cylindrical explosions and implosions (2D Riemann problems of
    a disc at rest in a gas at rest) in boxes of uneven sizes.

    Instance i: NX ~ U{n_lo..n_hi} and NY ~ U{n_lo..n_hi} square cells of
    side h on [0, NX h] x [0, NY h]; a disc of radius r ~ U[0.15, 0.35]
    min(Lx, Ly) centred at (U[0.4, 0.6] Lx, U[0.4, 0.6] Ly); rho and p
    log-uniform in [0.1, 10] inside and outside, redrawn (from the same
    stream) while the density ratio across the disc edge exceeds 20 -- the
    scheme has no positivity limiter, and larger ratios on the staircase edge
    of a disc drive the first step to a negative pressure; transmissive
    boundaries; t_end = 0.2 min(Lx, Ly) / max(c_in, c_out).
    Returns a dict of arrays and the number of redraws."""
    rng = np.random.Generator(np.random.Philox(seed))
    NX = np.zeros(count, dtype=np.int64); NY = np.zeros(count, dtype=np.int64)
    r = np.zeros(count); cx = np.zeros(count); cy = np.zeros(count)
    rho = np.zeros((count, 2)); p = np.zeros((count, 2))     # inside, outside
    redraws = 0
    i = 0
    while i < count:
        nx, ny = (int(v) for v in rng.integers(n_lo, n_hi + 1, size=2))
        fr, fx, fy = rng.uniform(0.15, 0.35), rng.uniform(0.4, 0.6), rng.uniform(0.4, 0.6)
        ri, ro, pi, po = np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=4))
        if max(ri / ro, ro / ri) > 20.0:
            redraws += 1
            continue
        NX[i], NY[i] = nx, ny
        L = min(nx, ny) * h
        r[i], cx[i], cy[i] = fr * L, fx * nx * h, fy * ny * h
        rho[i] = (ri, ro); p[i] = (pi, po)
        i += 1
    c = np.sqrt(gamma * p / rho)
    T = 0.2 * np.minimum(NX, NY) * h / c.max(axis=1)
    return dict(NX=NX, NY=NY, h=h, r=r, cx=cx, cy=cy, rho=rho, p=p, t_end=T, gamma=gamma), redraws


def explosion_instance(params: dict, i: int):
    """Problem description and initial state [4][NY][NX] of instance i of an
    explosion batch (transmissive boundaries)."""
    nx, ny, h = int(params["NX"][i]), int(params["NY"][i]), params["h"]
    g = params["gamma"]
    x = centers(0.0, nx * h, nx)[None, :]
    y = centers(0.0, ny * h, ny)[:, None]
    inside = (x - params["cx"][i]) ** 2 + (y - params["cy"][i]) ** 2 < params["r"][i] ** 2
    rho = np.where(inside, params["rho"][i, 0], params["rho"][i, 1])
    p = np.where(inside, params["p"][i, 0], params["p"][i, 1])
    z = np.zeros((ny, nx))
    prob = _base(2, [nx, ny], [0.0, 0.0], [nx * h, ny * h], [BC_TRANSMISSIVE] * 2, [BC_TRANSMISSIVE] * 2,
                 float(params["t_end"][i]), f"explosion_{i}", gamma=g)
    return prob, prim_to_cons(g, rho, [z, z], p)


def riemann_instance(params: dict, i: int):
    """Problem description and initial state of instance i of a batch."""
    n = int(params["N"][i])
    return riemann_1d(n, tuple(params["WL"][i]), tuple(params["WR"][i]), float(params["t_end"][i]),
                      gamma=params["gamma"], name=f"riemann_{i}")
