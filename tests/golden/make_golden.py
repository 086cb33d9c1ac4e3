"""Writes the stored expected values under tests/golden/ from the FP64 oracle only.

    python tests/golden/make_golden.py

c1_ed.txt: the lowest 12 eigenvalues (cm^-1) of the seeded 4-mode Hamiltonian (seed 0, d = 6),
by dense exact diagonalisation of its 1296 x 1296 matrix (Eq. sum_of_tp)."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import network as N  # noqa: E402
from paper_2512_15875_gb300 import inputs as I  # noqa: E402


def main():
    w = I.make_workload("c1", seed=0)
    ev = np.linalg.eigvalsh(N.dense_hamiltonian(w.ham))[:12]
    with open(os.path.join(HERE, "c1_ed.txt"), "w") as f:
        f.write("# lowest 12 eigenvalues (cm^-1) of the 4-mode workload, seed 0, d = 6, dense ED\n")
        for e in ev:
            f.write(f"{e:.12f}\n")


if __name__ == "__main__":
    main()
