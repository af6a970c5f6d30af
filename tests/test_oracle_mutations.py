"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each case patches one plausible error into a copy of an oracle routine and
re-runs the check that is meant to catch it."""
import math

import numpy as np

from oracle import ifeast_oracle as orc
from paper_1706_00692_gb300 import inputs


def _gl_half_without_half(nc, emin, emax):
    c, r = 0.5 * (emin + emax), 0.5 * (emax - emin)
    x, g = np.polynomial.legendre.leggauss(nc)
    th = 0.5 * math.pi * (1.0 - x)
    return c + r * np.exp(1j * th), g * r * np.exp(1j * th)      # dropped factor 1/2


def test_dropped_weight_factor_is_caught():
    z, w = _gl_half_without_half(8, 2.0, 5.0)
    assert abs(orc.filter_rho(np.array([3.5]), z, w, True)[0] - 1.0) > 0.5


def test_wrong_trapezoid_offset_is_caught():
    N, t = 8, 1.2
    th = 2.0 * math.pi * np.arange(N) / N                          # nodes not offset by 1/2
    z, w = 1.0 + 2.0 * np.exp(1j * th), 2.0 * np.exp(1j * th) / N
    val = orc.filter_rho(np.array([1.0 + 2.0 * t]), z, w, False)[0]
    assert abs(val - 1.0 / (1.0 + t ** N)) > 1e-3


def test_sign_error_in_shift_is_caught():
    A = inputs.laplacian((10, 9))
    ev = orc.laplacian_closed_form_eigs((10, 9))
    emin, emax = 0.0, 0.5 * (ev[4] + ev[5])
    Ad = A.to_scipy().toarray()
    z, w = orc.contour_nodes(orc.GL_HALF, 8, emin, emax)
    X = inputs.initial_subspace(A.n, 7, 0)
    bad = np.zeros(X.shape)
    for zk, wk in zip(z, w):                                       # (A - zI) instead of (zI - A)
        bad += (wk * np.linalg.solve(Ad - zk * np.eye(A.n), X.astype(complex))).real
    ref = orc.filter_step_spectral(Ad, X, z, w, True)
    assert np.abs(bad - ref).max() > 0.1 * np.abs(ref).max()


def test_missing_conjugate_in_gmres_dot_is_caught():
    n = 15
    g = np.random.default_rng(5)
    M = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)) + 4 * np.eye(n)
    b = g.standard_normal(n).astype(np.complex128)
    k = 5
    V = np.zeros((k + 1, n), complex)
    H = np.zeros((k + 1, k), complex)
    V[0] = b / np.linalg.norm(b)
    for s in range(k):
        wv = M @ V[s]
        for l in range(s + 1):
            H[l, s] = np.sum(V[l] * wv)                            # no conjugate
            wv = wv - H[l, s] * V[l]
        H[s + 1, s] = np.linalg.norm(wv)
        V[s + 1] = wv / H[s + 1, s]
    rhs = np.zeros(k + 1, complex)
    rhs[0] = np.linalg.norm(b)
    y = V[:k].T @ np.linalg.lstsq(H, rhs, rcond=None)[0]
    good = orc.gmres(lambda x: M @ x, b, k)
    assert np.linalg.norm(b - M @ y) > 1.01 * good["res_est"] or np.abs(y - good["y"]).max() > 1e-6
