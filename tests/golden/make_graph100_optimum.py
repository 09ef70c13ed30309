#!/usr/bin/env python3
"""Write graph100_optimum.txt: the optimum of the 100-node graph instance (p = 5) by the oracle's brute force.

The instance is paper_shape_instance("graph100"): a connected random graph with n = m = 100 nodes and 200 edges,
weights uniform in [1, 100], all-pairs shortest-path distances, seed 0 -- the shape of OR-Library pmed1
(Section 6, Table 1).  Every one of the C(100, 5) = 75,287,520 open sets is costed by the oracle's direct
objective (Section 1, Eqs. 1-3) in oracle_brute_force; nothing here calls the CUDA library.

    python tests/golden/make_graph100_optimum.py
"""

import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1610_10061_gb300.inputs import paper_shape_instance  # noqa: E402


def main():
    w = paper_shape_instance("graph100")
    d, p = w["d"], w["p"]
    n, m = d.shape
    cost, best = oracle.brute_force_c(d, p)
    with open(os.path.join(HERE, "graph100_optimum.txt"), "w") as fh:
        fh.write("# Optimum of the 100-node graph instance (paper_shape_instance('graph100'): n = m = 100, 200 edges,\n"
                 "# weights U[1,100], APSP distances, seed 0; the shape of OR-Library pmed1, Section 6 Table 1)\n"
                 f"# for p = {p}: all C({m}, {p}) = {math.comb(m, p)} open sets costed by the oracle's direct\n"
                 "# objective (Section 1, Eqs. 1-3), oracle_brute_force; written by make_graph100_optimum.py.\n"
                 "# [cost] the optimum; [open] its facilities (0-based, ascending; ties: lexicographically first).\n")
        fh.write(f"[cost]\n{cost}\n[open]\n{' '.join(str(j) for j in best)}\n")
    print(cost, best)


if __name__ == "__main__":
    main()
