"""Write lattice_contacts.txt: every lattice placement of two unit solids
whose interiors overlap (exact separating-axis test), with the strict
intersection predicate's verdict computed by the CPU oracle.

The placements the predicate reports as not intersecting are the contacts
realised only through coincident edges and vertices, which the strict
reading of the paper's piercing (Sec. 3.2; tangential contact excluded,
Sec. 3.6) does not count.  Run from the repository root:
    python tests/golden/make_lattice_contacts.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))                  # tests/ (cases)
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))  # repository root

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from cases import lattice_case_sets, sat_overlap  # noqa: E402


def rows():
    A, B, cand, meta = lattice_case_sets()
    verdict = oracle.join(A, B, cand, tier=1)
    out = []
    for k, (i, j) in enumerate(cand):
        va, ta = A.mesh(int(i))
        vb, tb = B.mesh(int(j))
        if sat_overlap(va.astype(np.int64), ta, vb.astype(np.int64), tb):
            na, nb, o = meta[k]
            out.append((na, nb, int(o[0]), int(o[1]), int(o[2]), int(verdict[k])))
    return out


def main():
    oracle.build()
    with open(os.path.join(HERE, "lattice_contacts.txt"), "w") as f:
        f.write("# Lattice placements (B = A's unit solid shifted by an integer offset in\n"
                "# [-3, 3]^3) whose interiors overlap by the exact separating-axis test, and\n"
                "# the strict intersection predicate's verdict from the CPU oracle (1 = pair\n"
                "# reported).  0 rows are contacts through coincident edges and vertices only.\n"
                "# Written by tests/golden/make_lattice_contacts.py.\n"
                "# shape_a shape_b dx dy dz intersects\n")
        for r in rows():
            f.write("%s %s %d %d %d %d\n" % r)


if __name__ == "__main__":
    main()
