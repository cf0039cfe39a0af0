"""Writes tests/golden/pair_integrals.txt: brute-force values of
(1/4pi) int_P int_Q 1/|x-y| for touching and separated triangle pairs.

Calls only oracle.bruteforce (nested adaptive quadrature with a closed-form
innermost line integral), never the CUDA path or the oracle's own rules.
Run:  python tests/golden/make_pair_golden.py   (several minutes)
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import bruteforce  # noqa: E402

A = [0.0, 0.0, 0.0]
B = [1.0, 0.0, 0.0]
C = [0.3, 0.9, 0.0]
D = [0.2, -0.4, 0.7]
E = [-0.6, 0.1, 0.5]
F = [0.5, 0.0, 1.0]
CASES = [
    # name, type, P (shared vertices first, in the same order in Q), Q
    ("vertex_skew", "vertex", [A, B, C], [A, D, E]),
    ("vertex_coplanar", "vertex", [A, B, C], [A, [-1.0, 0.2, 0.0], [-0.4, -0.8, 0.0]]),
    ("edge_skew", "edge", [A, B, C], [A, B, D]),
    ("edge_right_angle", "edge", [A, B, [0.5, 1.0, 0.0]], [A, B, F]),
    ("far_offset", "far", [A, B, C], [[0.5, 2.0, 0.3], [1.5, 2.0, 0.3], [0.8, 2.9, 0.3]]),
]


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pair_integrals.txt")
    with open(out, "w") as f:
        f.write("# (1/4pi) int_P int_Q 1/|x-y|: brute force by oracle/bruteforce.py\n")
        f.write("# (scipy nested adaptive quadrature, closed-form innermost line integral,\n")
        f.write("# epsabs 1e-12, epsrel 1e-11).  Generated by tests/golden/make_pair_golden.py.\n")
        f.write("# name type P(9) Q(9) value\n")
        for name, typ, P, Q in CASES:
            v = bruteforce.pair_integral(np.array(P), np.array(Q))
            nums = " ".join(repr(float(c)) for c in np.ravel(P)) + " " + " ".join(repr(float(c)) for c in np.ravel(Q))
            f.write(f"{name} {typ} {nums} {v!r}\n")
            f.flush()
            print(name, v, flush=True)


if __name__ == "__main__":
    main()
