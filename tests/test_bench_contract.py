"""CPU checks of the benchmark's constants against the oracle."""
import numpy as np

import bench
from oracle import oracle as orc


def test_algorithmic_flop_table_matches_oracle_counts():
    for dim in (1, 2, 3):
        prob = dict(dim=dim, n=[8] * dim, lo=[0] * dim, hi=[1] * dim, bc_lo=[0] * dim, bc_hi=[0] * dim)
        U = np.array([1.0] + [0.3] * dim + [3.0])
        U6 = np.stack([U * (1 + 0.1 * m) for m in range(6)])
        c = orc.count_cell(prob, 0, U).sum()
        fu, s1 = orc.count_face(prob, 0, U6, 1e300)
        fw, s2 = orc.count_face(prob, 0, U6, -1.0)
        assert s1 and not s2
        assert bench.ALG_FLOPS[dim] == (c, fu.sum(), fw.sum())
        ce = orc.count_cell(prob, 0, U, essential=True).sum()
        fue, _ = orc.count_face(prob, 0, U6, 1e300, essential=True)
        fwe, _ = orc.count_face(prob, 0, U6, -1.0, essential=True)
        assert bench.ALG_FLOPS_ESSENTIAL[dim] == (ce, fue.sum(), fwe.sum())


def test_essential_counts_leave_out_only_folded_and_structural_operations():
    """One Euler cell: the essential count drops only the first sum of
    |u|^2 = 0 + u u, which starts from a known zero."""
    prob = dict(dim=1, n=[8], lo=[0], hi=[1], bc_lo=[0], bc_hi=[0])
    U = np.array([1.0, 0.3, 3.0])
    for essential in (False, True):
        c = orc.count_cell(prob, 0, U, essential=essential)
        assert c[3] == 1                      # one square root (sound speed) either way
    w = orc.count_cell(prob, 0, U)
    e = orc.count_cell(prob, 0, U, essential=True)
    assert np.all(e <= w) and e.sum() == w.sum() - 1 and e[0] == w[0] - 1


def test_sweep_flops_formula():
    f = bench.sweep_flops(2, [10, 4], 0, 0)
    fc, fu, fw = bench.ALG_FLOPS[2]
    assert f == 40 * (fc + 8) + 44 * fu


def test_direction_dependent_cell_flops():
    """The per-cell operations a sweep that reads the stage's primitives is
    credited with: the physical flux along the sweep (dim products u_n m_k,
    the pressure sum, E + p and its product with u_n) and the two acoustic
    eigenvalues u_n -+ c.  The rest of the oracle's cell count (velocity,
    |u|^2, p, c, H) is at least what those primitives take."""
    for dim in (1, 2, 3):
        assert bench.ALG_FLOPS_CELL_DIR[dim] == dim + 1 + 2 + 2
        prob = dict(dim=dim, n=[8] * dim, lo=[0] * dim, hi=[1] * dim, bc_lo=[0] * dim, bc_hi=[0] * dim)
        U = np.array([1.0] + [0.3] * dim + [3.0])
        c = orc.count_cell(prob, 0, U)
        # primitives: dim divisions (velocity), one square root (c) and at
        # least the dim products of |u|^2 remain outside the credited part
        assert c.sum() - bench.ALG_FLOPS_CELL_DIR[dim] >= dim + 1 + dim
        assert c[2] >= dim and c[3] == 1
    assert bench.reads_prims("fp64", 2, 0) and not bench.reads_prims("fp64", 2, 1)
    assert not bench.reads_prims("fp32", 2, 0) and not bench.reads_prims("fp64", 1, 0)
    f = bench.sweep_flops(2, [10, 4], 0, 0, prims_read=True)
    assert f == 40 * (bench.ALG_FLOPS_CELL_DIR[2] + 8) + 44 * bench.ALG_FLOPS[2][1]
