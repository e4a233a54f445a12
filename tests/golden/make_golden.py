"""Writes the stored expected values under tests/golden/ by calling only oracle/.

The paper prints no worked numerical example of an element matrix (its only
numbers are timings and the Amdahl tables of Sec. 4), so the stored fixtures
are oracle regression values on small seeded cases: they detect drift of the
oracle's arithmetic between commits.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2207_00280_gb300 import workloads as wl  # noqa: E402

CASES = {
    # name: (dim, p, K, q, curved, kappa seed, elements)
    "oracle_2d_p2_K4": (2, 2, 4, 3, False, 31, [0, 5, 15]),
    "oracle_3d_p2_K3_curved": (3, 2, 3, 3, True, 32, [0, 13, 26]),
}


def compute(name):
    dim, p, K, q, curved, seed, elems = CASES[name]
    knots = [wl.open_uniform_knots(K, p)] * dim
    P = oracle.Patch(knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, seed)
    G = wl.curved_map_jacobian(knots, q) if curved else None
    Km, Mm = P.classical(np.array(elems), kappa=kappa, G=G)
    return elems, Km, Mm


def main():
    for name in CASES:
        elems, Km, Mm = compute(name)
        path = os.path.join(HERE, name + ".txt")
        with open(path, "w") as f:
            f.write(f"# {name}: oracle classical element matrices (K then M), elements {elems}\n")
            f.write("# written by tests/golden/make_golden.py (oracle only)\n")
            for e in range(len(elems)):
                for mat in (Km[e], Mm[e]):
                    for row in mat:
                        f.write(" ".join(f"{v:.17e}" for v in row) + "\n")
        print("wrote", path)


if __name__ == "__main__":
    main()
