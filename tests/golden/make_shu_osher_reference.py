"""Write shu_osher_rho_ref400.txt: the density of the shock / entropy-wave
interaction (Sec. 4.4; the workload's shifted form on [-5, 5]) at t = 1.8,
computed by the FP64 oracle on 3200 cells and averaged over groups of eight
cells onto the 400-cell grid.  Sec. 4.4 compares against a 3200-point
high-resolution run; here the reference is the present method's own oracle.

Usage: python tests/golden/make_shu_osher_reference.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as orc  # noqa: E402
from paper_1908_02464_gb300 import problems as P  # noqa: E402

OUT = os.path.join(HERE, "shu_osher_rho_ref400.txt")


def reference():
    prob, U = P.shu_osher(3200)
    U = np.ascontiguousarray(U)
    st, t, k = orc.advance(prob, U, 0.0, prob["t_end"])
    assert st == 0 and t == prob["t_end"]
    return U[0].reshape(400, 8).mean(axis=1), k


def main():
    rho, k = reference()
    with open(OUT, "w") as f:
        f.write("# Shu-Osher density at t = 1.8 (Sec. 4.4, domain [-5, 5], jump at x = -4), FP64 oracle on\n")
        f.write(f"# 3200 cells ({k} RK3 steps, CFL 0.5, LLF, hybrid on), averaged over 8 cells onto 400 cells.\n")
        f.write("# Written by tests/golden/make_shu_osher_reference.py (oracle only).\n")
        for v in rho:
            f.write(f"{v:.17e}\n")


if __name__ == "__main__":
    main()
