"""Writes tests/golden/lap3d64_window.txt from the oracle only: the eigenvalues
of the 64^3 7-point Laplacian + U[0,1) potential (potential seed 1, the bench's
matrix) nearest the interior window, and the window itself.

Run from the repository root (about 7 minutes on 8 cores: one sparse LU of the
shifted matrix in nested-dissection order, then shift-invert Lanczos):

    python tests/golden/make_lap3d64_window.py

Window rule: a first window of ~50 eigenvalues is
[lam_L(1001) + 0.5, lam_L(1051) + 0.5] from the pure Laplacian's closed-form
spectrum shifted by the potential's mean; each endpoint is moved to the
midpoint of the widest spectral gap of A whose midpoint lies within 1e-3 of
that first endpoint, so that Ritz values of the eigenvectors just outside
stay clear of the endpoints.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ifeast_oracle as orc  # noqa: E402
from paper_1706_00692_gb300 import inputs  # noqa: E402  (seeded matrix generator only)

HERE = os.path.dirname(os.path.abspath(__file__))
N = 64
K_NEAR = 100


def window_from_gaps(lam, target, reach=1e-3):
    g = np.diff(lam)
    mid = 0.5 * (lam[1:] + lam[:-1])
    ok = np.abs(mid - target) <= reach
    if not ok.any():
        raise ValueError("no gap near the target")
    k = np.argmax(np.where(ok, g, -1.0))
    return float(mid[k])


def main():
    A = inputs.add_diagonal_fast(inputs.laplacian((N, N, N)), inputs.random_potential(N ** 3, 1))
    evL = orc.laplacian_closed_form_eigs((N, N, N))
    lo_t, hi_t = evL[1000] + 0.5, evL[1050] + 0.5
    centre = 0.5 * (lo_t + hi_t)
    lam, _, res = orc.eigenpairs_near(A.to_scipy(), centre, K_NEAR,
                                      orc.grid_nested_dissection((N, N, N)))
    emin, emax = window_from_gaps(lam, lo_t), window_from_gaps(lam, hi_t)
    # completeness: the K_NEAR eigenvalues nearest the centre reach past both ends
    assert lam.min() < emin and lam.max() > emax
    assert max(abs(lam.min() - centre), abs(lam.max() - centre)) > max(centre - emin, emax - centre)
    inside = (lam > emin) & (lam < emax)
    with open(os.path.join(HERE, "lap3d64_window.txt"), "w") as f:
        f.write("# Eigenvalues of A = L + V nearest the interior window: L the 64^3 7-point Dirichlet\n")
        f.write("# Laplacian, V = diag(U[0,1)) from PCG64(1) (the bench's matrix), computed by the\n")
        f.write("# oracle's shift-invert Lanczos (tests/golden/make_lap3d64_window.py). Column 1:\n")
        f.write("# eigenvalue, column 2: residual ||A x - lam x|| (an exact eigenvalue lies within it),\n")
        f.write("# column 3: 1 if inside the window. The window endpoints are the midpoints of the\n")
        f.write("# widest gaps within 1e-3 of the first window [lam_L(1001) + 0.5, lam_L(1051) + 0.5].\n")
        f.write(f"# window {emin:.17e} {emax:.17e}\n")
        f.write(f"# inside {int(inside.sum())}\n")
        for v, r, i in zip(lam, res, inside):
            f.write(f"{v:.17e} {r:.3e} {int(i)}\n")
    print(f"window ({emin:.10f}, {emax:.10f}), {int(inside.sum())} inside, max residual {res.max():.2e}")


if __name__ == "__main__":
    main()
