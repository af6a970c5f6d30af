"""Host logic of the benchmark's measurement: algorithmic bytes of the Lanczos
step, the per-class statistics of sampled kernel timing, and the roofline entry
(which class is dominant, achieved bandwidth, fraction of the peak)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_1706_00692_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def wl():
    return inputs.workload_lap3d_64_interior()


def test_step_bytes_lap3d_64(wl):
    # read w_{s-1}, v_{s-1}; write v_s, w_s (4 x n x m0 x 4 B) + CSR (4 (n+1) + 8 nnz)
    n, m0, nnz = 262144, 80, 1810432
    assert bench.step_bytes(wl, 4) == 4 * n * m0 * 4 + 4 * (n + 1) + 8 * nnz == 351076356


def test_kernel_stats_from_sampled_timing():
    ktimes = {"lanczos_step": (10, 0.9), "rr_eig": (3, 15.0)}
    klaunch = {"lanczos_step": 80, "rr_eig": 3}
    ks = bench.kernel_stats(ktimes, klaunch)
    assert ks["lanczos_step"] == (80, 10, pytest.approx(0.09))
    assert ks["rr_eig"] == (3, 3, pytest.approx(5.0))


def test_roofline_of_the_dominant_step_kernel(wl):
    ks = {"lanczos_step": (9000, 1000, 0.09), "lanczos_quadrature": (7, 7, 16.0)}
    r = bench.lanczos_roofline(ks, wl, 6795.8, "measured")
    assert r["launches"] == 9000 and r["launches_timed"] == 1000
    assert r["achieved"] == pytest.approx(351076356 / 90e-6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6795.8)
    assert r["traffic"] == bench.ELL_STEP_TRAFFIC_LAP3D64
    # another class dominating: no step-kernel roofline
    ks2 = {"lanczos_step": (10, 10, 0.09), "gmres_spmm_dot": (300, 300, 17.0)}
    assert bench.lanczos_roofline(ks2, wl, 6795.8, "measured") is None
