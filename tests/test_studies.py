"""Host-side pins of the side studies in bench.py (accuracy slope, deflection
perturbation PDF).  CPU only.

* Katz et al.'s Eq. 13 (and the paper's modified numerator, Sec. 2.3) is a
  probability density: it integrates to 1 over the plane.
* Far from the typical deflection the perturbation is that of the single
  nearest unit-mass lens, so P(|alpha|/phi_0 > u) -> 1/u^2 for lenses of
  density kappa_*/pi: the density tends to 1/(pi u^4).  This limit does not
  come from the formula, so it pins the numerics of the integral.
* The width grows with the number of lenses (Sec. 2.3).
* The log-binned RMS and the log-log fit recover a known power law.
"""
import numpy as np
import pytest

import bench


@pytest.mark.parametrize("n", [1e2, 1e4, 1e6])
@pytest.mark.parametrize("c", [1.454, 3.05])
def test_katz_density_is_normalised(n, c):
    u = np.linspace(0.0, 60.0, 1201)
    d = bench.katz_density(u, n, c)
    total = np.trapezoid(d * 2 * np.pi * u, u)
    assert 0.999 <= total <= 1.0005, total


@pytest.mark.parametrize("n", [1e2, 1e4])
def test_katz_tail_is_the_nearest_lens_tail(n):
    # u = 40: far in the tail, still inside the range the quadrature resolves
    # (beyond u ~ 50 the tail is a 1e-8 remainder of an oscillating integral)
    d = bench.katz_density(np.array([40.0]), n, 1.454)[0]
    assert abs(d * np.pi * 40.0 ** 4 - 1.0) < 0.05, d * np.pi * 40.0 ** 4


def test_katz_width_grows_with_lens_count():
    u = np.linspace(0.0, 40.0, 801)
    med = []
    for n in (1e2, 1e3, 1e4, 1e6):
        d = bench.katz_density(u, n, 1.454)
        cdf = np.cumsum(d * 2 * np.pi * u) * (u[1] - u[0])
        med.append(u[np.searchsorted(cdf, 0.5)])
    assert all(a < b for a, b in zip(med, med[1:])), med


def test_loglog_slope_of_a_power_law():
    x = np.logspace(0, 4, 50)
    assert bench.loglog_slope(x, 3.0 * x ** (-2.0 / 3.0)) == pytest.approx(-2.0 / 3.0, abs=1e-12)


def test_log_binned_rms_recovers_the_error_slope():
    rng = np.random.default_rng(4)
    n = np.maximum(1, np.round(np.exp(rng.uniform(np.log(5), np.log(5000), 400000))))
    err = n ** -0.75 * rng.standard_normal(n.size)
    x, y, w = bench.log_binned_rms(n, err, nbins=300, min_count=30)
    assert len(x) > 100
    fit = x >= 10
    assert bench.loglog_slope(x[fit], y[fit], w[fit]) == pytest.approx(-0.75, abs=0.02)


@pytest.mark.gpu
def test_accuracy_replay_small_case():
    """The accuracy replay end to end on a small case (64^2 map, 300 lenses,
    a 2e8-ray brute-force reference, interpolated maps of 1e6 ... 1.6e7
    rays): lattice sampling error falls with the ray count, so the fitted
    slope is negative, and the interpolated map of the reference's rays
    stays close to the brute force."""
    from gpu_common import require_gpu
    torch = require_gpu()
    from paper_2204_10871_gb300 import irs, lensgen
    out = bench.accuracy_replay(torch, irs, lensgen, ks=0.4, S=8.0, npix=64, n_star=300, ref_rays=2.0e8,
                                test_rays=(1.0e6, 4.0e6, 1.6e7), reference="brute", ref_chunk_rays=5.0e7,
                                fit_min=5.0)
    assert out["reference"]["method"] == "brute" and out["reference"]["bands"] >= 2
    assert out["reference"]["interp_same_rays_rel_rms"] < 1e-3
    assert len(out["maps"]) == 3
    errs = [mp["rel_rms_all_pixels"] for mp in out["maps"]]
    assert errs[0] > errs[1] > errs[2], errs
    assert -1.2 < out["slope_all_maps"] < -0.3, out["slope_all_maps"]
