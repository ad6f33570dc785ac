"""Writes the regression fixtures under tests/golden/ from the CPU oracle only.

fig1_counts.json: the synthetic operand pairs of the paper's Fig. 1 (n = 512,
tau = 1e-8; pair A: A_ij = exp(-|i-j|), B_ij = exp(-2|i-j|); pair B:
A_ij = B_ij = 1/|i-j|^3 off the diagonal). The paper shows these only as a plot of the
truncated product space, with no numbers, so the oracle's own per-tier test and cull
counts are frozen here as a regression fixture (not a paper value).

Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1011_3534_gb300 import workloads as W  # noqa: E402


def main():
    cases = []
    for pair in ("A", "B"):
        for leaf in (4, 16):
            A, B = W.fig1_pair(pair, 512)
            TA, TB = oracle.Tree(A, leaf), oracle.Tree(B, leaf)
            r = oracle.spamm(TA, TB, 1e-8, product=False, stats=True)
            cases.append(dict(pair=pair, n=512, leaf=leaf, tau=1e-8,
                              leaf_triples=r["count"], tested=r["stats"].tested,
                              culled=r["stats"].culled))
    out = dict(source="Fig. 1 operand pairs (Sec. II); counts written by the CPU oracle",
               cases=cases)
    with open(os.path.join(HERE, "fig1_counts.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
