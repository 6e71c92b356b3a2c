"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
Each output file names the cell recipe and the oracle routine that produced it.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.exact import exact_eigs  # noqa: E402
from oracle.planewave import PWOperator  # noqa: E402
from synth import config_cell  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def write_exact(name: str, nkeep: int):
    cell = config_cell(name)
    w = exact_eigs(PWOperator.from_cell(cell))
    path = os.path.join(HERE, "%s_exact_eigs.txt" % name)
    with open(path, "w") as f:
        f.write("# lowest %d eigenvalues (Ha) of the pencil (H, S) of synthetic cell '%s'\n" % (nkeep, name))
        f.write("# (npw=%d, nproj=%d), from oracle.exact.exact_eigs: dense H and S of Section 2.1,\n"
                % (cell.npw, cell.nproj))
        f.write("# Cholesky reduction, self-written cyclic Jacobi.  Written by tests/golden/make_golden.py\n")
        for x in w[:nkeep]:
            f.write("%.17e\n" % x)
    print("wrote", path)


if __name__ == "__main__":
    write_exact("nc24", 48)
