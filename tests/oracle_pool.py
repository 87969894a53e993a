"""Oracle runs of batch instances in worker processes.

The GPU tests hold a CUDA context, so the pool is started with `spawn`
(a forked child of a CUDA process can hang).  Workers regenerate the
seeded batch description themselves (cached per process) and return only
what the tests compare: status, time, steps and the final density."""
from __future__ import annotations

import functools
import os
from multiprocessing import get_context

import numpy as np


@functools.lru_cache(maxsize=4)
def _params(kind: str, count: int, seed: int):
    from paper_1908_02464_gb300 import problems as P
    if kind == "riemann":
        return P.riemann_batch_params(count, seed=seed)[0]
    return P.explosion_batch_params(count, seed=seed)[0]


def run_instance(job):
    """job = (kind, count, seed, i, max_steps[, pert]): the oracle's run of
    instance i to its end time, or to max_steps steps; with pert, from the
    initial state perturbed by one ulp at random (seed pert) in every value."""
    from oracle import oracle as orc
    from paper_1908_02464_gb300 import problems as P
    kind, count, seed, i, max_steps = job[:5]
    par = _params(kind, count, seed)
    prob, U = (P.riemann_instance if kind == "riemann" else P.explosion_instance)(par, i)
    if len(job) > 5 and job[5] is not None:
        rng = np.random.default_rng(job[5])
        U = np.ascontiguousarray(U * (1.0 + 2.220446049250313e-16 * rng.choice([-1.0, 0.0, 1.0], size=U.shape)))
    st, t, k = orc.advance(prob, U, 0.0, prob["t_end"], max_steps=max_steps)
    return i, st, t, k, U[0].copy()


def check_runs(kind: str, count: int, seed: int, st, steps, t, rho_gpu, sample, label: str,
               cap: float = 1e-4):
    """Batch instances against the oracle.  Every instance in `sample` takes
    the oracle's status, steps and end time, and its final density agrees
    in L1 to 1e-10, or -- where a hybrid flag sits at its threshold during
    the run, so that rounding decides between the linear and the WENO flux --
    to ten times the oracle's own run-to-run change under one-ulp
    perturbations of the initial state (5 or 16 draws), capped at `cap`;
    such instances are recorded (tests/parity_log.py).  Over runs of
    hundreds to thousands of steps a few percent of the instances meet such
    a face; the oracle's own sensitivity then reaches a few 1e-6, hence the
    cap of 1e-4 (an error in the scheme would show at the 1e-2 level).
    Returns the L1 values."""
    from tests import parity_log
    res = {r[0]: r for r in run_many([(kind, count, seed, i, 10 ** 9) for i in sample])}
    l1 = {}
    for i in sample:
        _, so, to, ko, rho = res[i]
        assert so == st[i] and ko == steps[i] and to == t[i], (i, so, st[i], ko, steps[i])
        l1[i] = float(np.mean(np.abs(rho_gpu[i] - rho)))
    loose = [i for i in sample if l1[i] > 1e-10]
    if loose:
        # whether a perturbation moves a face across the threshold is a
        # matter of chance: five draws, then eleven more where five fall short
        pert = {}
        for r in run_many([(kind, count, seed, i, 10 ** 9, p) for i in loose for p in range(1, 6)]):
            pert.setdefault(r[0], []).append(r[4])
        kap = {i: max(float(np.mean(np.abs(q - res[i][4]))) for q in pert[i]) for i in loose}
        more = [i for i in loose if l1[i] > 10.0 * kap[i]]
        if more:
            for r in run_many([(kind, count, seed, i, 10 ** 9, p) for i in more for p in range(6, 17)]):
                kap[r[0]] = max(kap[r[0]], float(np.mean(np.abs(r[4] - res[r[0]][4]))))
        for i in loose:
            parity_log.bar(l1[i], 1.0, 1e-10, lambda k=kap[i]: k, f"{label} instance {i}, L1(rho)", cap=cap)
    for i in sample:
        if i not in loose:
            parity_log.record(f"{label} instance {i}, L1(rho)", "strict", l1[i])
    return l1


def run_many(jobs, procs: int | None = None):
    procs = procs or min(16, os.cpu_count() or 1)
    with get_context("spawn").Pool(procs) as pool:
        return pool.map(run_instance, jobs, chunksize=max(1, len(jobs) // (4 * procs)))


def stratified(sizes: np.ndarray, ok: np.ndarray, k: int) -> list[int]:
    """k instances spread evenly over the size order, among those with ok."""
    order = [int(i) for i in np.argsort(sizes, kind="stable") if ok[i]]
    picks = np.linspace(0, len(order) - 1, min(k, len(order))).round().astype(int)
    return sorted({order[p] for p in picks})
