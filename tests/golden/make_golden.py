"""Writes the stored expected values under tests/golden/ from the oracle only.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ifeast_oracle as orc  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    ev = orc.laplacian_closed_form_eigs((50, 50))[:11]
    with open(os.path.join(HERE, "lap2d_50x50_lowest11.txt"), "w") as f:
        f.write("# 11 lowest eigenvalues of the 2D 5-point Dirichlet Laplacian on a 50x50 grid,\n")
        f.write("# lambda_{p,q} = (2-2cos(p pi/51)) + (2-2cos(q pi/51)) (textbook closed form).\n")
        f.write("# The 10 lowest are the wanted pairs of the 50x50 workload; the 11th fixes the\n")
        f.write("# interval's upper end (lambda_10 + lambda_11)/2.\n")
        for v in ev:
            f.write(f"{v:.17e}\n")


if __name__ == "__main__":
    main()
