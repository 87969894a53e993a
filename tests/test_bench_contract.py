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


def test_sweep_flops_formula():
    f = bench.sweep_flops(2, [10, 4], 0, 0)
    fc, fu, fw = bench.ALG_FLOPS[2]
    assert f == 40 * (fc + 8) + 44 * fu
