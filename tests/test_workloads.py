"""Host-side checks of the synthetic workloads the bench and the CLI use: the
interval endpoints sit in spectral gaps of the closed-form spectra, and the
counts, subspace sizes and names are the ones the bench reports."""
import numpy as np

from paper_1706_00692_gb300 import inputs


def test_fem3d_workload_interval_and_sizes():
    wl = inputs.workload_fem3d(64, 50, precision="fp32")
    ev = inputs.fem_q1_eigs((64, 64, 64))
    inside = (ev > wl.emin) & (ev < wl.emax)
    assert inside.sum() == wl.expected_count == 54
    assert wl.m0 == int(1.5 * 54) + 2 == 83
    # the upper endpoint is the midpoint of a gap of at least 1e-3 relative
    k = wl.expected_count
    assert ev[k] - ev[k - 1] > 1e-3 * ev[k]
    assert abs(wl.emax - 0.5 * (ev[k - 1] + ev[k])) <= 1e-12 * ev[k]
    assert wl.A.n == wl.B.n == 64 ** 3 and wl.A.nnz == wl.B.nnz
    assert (wl.A.rowptr == wl.B.rowptr).all() and (wl.A.colidx == wl.B.colidx).all()
    assert wl.name.startswith("fem3d_64^3_lowest54_m0_83")


def test_fem3d_small_gap_count():
    wl = inputs.workload_fem3d(12, 10, precision="fp64")
    ev = inputs.fem_q1_eigs((12, 12, 12))
    assert ((ev > wl.emin) & (ev < wl.emax)).sum() == wl.expected_count >= 10
    assert wl.precision == "fp64"


def test_lap3d_64_window_parameters():
    """The bench window of the 64^3 Laplacian + U[0,1) potential: its 56
    eigenvalues come from converged solves (the GPU test of the full-size
    workload checks them); here the window lies in the part of the spectrum
    the potential can reach (Weyl: every eigenvalue of L + V is within
    [lam_min(L), lam_max(L) + 1]) and the solver parameters are the bench's."""
    wl = inputs.workload_lap3d_64_interior()
    evL = inputs.laplacian_eigs((64, 64, 64))
    assert evL[0] < wl.emin < wl.emax < evL[-1] + 1.0
    assert wl.expected_count == 56
    assert wl.m0 == 80 and wl.nc == 8 and wl.rule == "trap_half"
    assert wl.inner == "minres" and wl.inner_iters == 1500 and wl.alpha == 3e-2
    assert np.isclose(wl.emax - wl.emin, 0.91001238 - 0.89754658)


def test_serving_requests_counts_match_dense_spectra():
    """Each request's interval holds exactly its stated count of eigenvalues of
    A = L + V (dense eigh on small requests): the potential is below a quarter
    of the gap at the upper end, so by Weyl's bounds no eigenvalue crosses it;
    m0 is a multiple of 4 at least the count; arrivals increase."""
    reqs = inputs.serving_requests(12, seed=77, n_min=200, n_max=1500)
    for r in reqs:
        ev = np.linalg.eigvalsh(r.A.to_scipy().toarray())
        inside = (ev > r.emin) & (ev < r.emax)
        assert inside.sum() == r.count
        assert r.m0 >= r.count and r.m0 % 4 == 0
        assert r.X0.shape == (r.A.n, r.m0)
    assert all(b.arrival > a.arrival for a, b in zip(reqs, reqs[1:]))


def test_lap3d64_window_comes_from_the_oracle_spectrum():
    """The 64^3 workload's window and count are those of the oracle-written
    golden file: the stored endpoints follow the file's gap rule applied to its
    eigenvalues, the constants equal them, 56 eigenvalues lie inside, the
    nearest ones outside are on both sides, and every stored eigenvalue has a
    residual small enough to fix it to 1e-11 relative (an exact eigenvalue lies
    within the residual norm; ten times tighter than the GPU comparison's 1e-10)."""
    import importlib.util
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    path = os.path.join(here, "lap3d64_window.txt")
    header = [l.split() for l in open(path) if l.startswith("# window")][0]
    emin, emax = float(header[2]), float(header[3])
    data = np.loadtxt(path)
    lam, res, ins = data[:, 0], data[:, 1], data[:, 2].astype(bool)
    spec = importlib.util.spec_from_file_location("mk", os.path.join(here, "make_lap3d64_window.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    evL = inputs.laplacian_eigs((64, 64, 64))
    assert mk.window_from_gaps(lam, evL[1000] + 0.5) == emin
    assert mk.window_from_gaps(lam, evL[1050] + 0.5) == emax
    assert inputs.LAP3D_64_WINDOW == (emin, emax)
    wl = inputs.workload_lap3d_64_interior()
    assert (wl.emin, wl.emax) == (emin, emax)
    assert ins.sum() == wl.expected_count == 56
    assert np.array_equal(ins, (lam > emin) & (lam < emax))
    assert (lam < emin).any() and (lam > emax).any()
    assert np.all(np.diff(lam) > 0)
    assert res.max() <= 1e-11 * lam.min()


def test_convdiff_workload_interval():
    """The 512 x 512 upwind convection-diffusion workload: the circle through 0
    and emax holds exactly the 40 lowest closed-form eigenvalues (all real),
    emax sits midway in the gap after the 40th, and the closed form matches a
    dense eigensolve on a small grid of the same generator."""
    import numpy as np
    from paper_1706_00692_gb300 import inputs
    wl = inputs.workload_convdiff(512)
    cf = inputs.upwind_convection_diffusion_eigs((512, 512), 10.0)
    assert wl.A.n == 512 * 512 and wl.m0 == 64 and wl.nonsym and wl.nonsym_correction
    c = r = wl.emax / 2
    assert int((np.abs(cf - c) < r).sum()) == 40 == wl.expected_count
    assert cf[39] < wl.emax < cf[40]
    assert abs(wl.emax - 0.5 * (cf[39] + cf[40])) <= 1e-12 * wl.emax
    small = inputs.upwind_convection_diffusion((12, 10), 10.0).to_scipy().toarray()
    ev = np.sort(np.linalg.eigvals(small).real)
    assert np.abs(ev - inputs.upwind_convection_diffusion_eigs((12, 10), 10.0)).max() <= 1e-10 * ev.max()
