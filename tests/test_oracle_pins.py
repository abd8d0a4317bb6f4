"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these uses the CUDA library.  Each test names the passage it checks
and the kind of mistake it would catch.
"""
import json
import os

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss
from scipy import integrate

import oracle
from paper_2204_10871_gb300 import lensgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- the sheet
def _quad_sheet(a1, a2, b1, b2, k, t1, t2):
    """Positive uniform rectangle deflection by adaptive 2-D quadrature of the
    Appendix A integrands, split at the field point so the 1/r singularity
    sits on sub-rectangle corners."""
    A = k / np.pi
    xs = [a1] + ([t1] if a1 < t1 < a2 else []) + [a2]
    ys = [b1] + ([t2] if b1 < t2 < b2 else []) + [b2]
    f1 = lambda y, x: (t1 - x) / ((t1 - x) ** 2 + (t2 - y) ** 2)
    f2 = lambda y, x: (t2 - y) / ((t1 - x) ** 2 + (t2 - y) ** 2)
    out = []
    for f in (f1, f2):
        tot = 0.0
        for i in range(len(xs) - 1):
            for j in range(len(ys) - 1):
                tot += integrate.dblquad(f, xs[i], xs[i + 1], ys[j], ys[j + 1],
                                         epsabs=1e-13, epsrel=1e-12)[0]
        out.append(A * tot)
    return out


@pytest.mark.parametrize("t", [(0.3, 0.2), (4.9, 1.9), (-2.5, -0.99), (7.0, 4.0), (1.0, -3.0),
                               (-3.0, 0.5), (5.0, 2.0)])
def test_sheet_closed_form_matches_quadrature(t):
    """Appendix A: the printed alpha_1, alpha_2 equal the defining double
    integrals (catches a dropped term, swapped corner or wrong sign)."""
    rect = (-3.0, 5.0, -1.0, 2.0)
    q = _quad_sheet(*rect, 0.4, *t)
    o = oracle.sheet_positive(*rect, 0.4, *t)
    assert abs(o[0] - q[0]) < 1e-11 and abs(o[1] - q[1]) < 1e-11


def test_sheet_divergence_curl():
    """A uniform sheet of density k has div(alpha) = 2k inside and 0 outside,
    and curl 0 (Poisson equation of the lens potential)."""
    rect = (-2.0, 3.0, -1.5, 1.0)
    k, h = 0.45, 1e-4
    f = lambda x, y: np.array(oracle.sheet_positive(*rect, k, x, y))
    for (x, y), inside in [((0.1, 0.2), True), ((2.7, -1.2), True), ((-1.9, 0.9), True),
                           ((4.0, 0.0), False), ((0.0, -3.0), False), ((-6.0, 5.0), False)]:
        dx = (f(x + h, y) - f(x - h, y)) / (2 * h)
        dy = (f(x, y + h) - f(x, y - h)) / (2 * h)
        div, curl = dx[0] + dy[1], dx[1] - dy[0]
        assert abs(div - (2 * k if inside else 0.0)) < 1e-6
        assert abs(curl) < 1e-6


def test_sheet_far_limit_and_centre():
    """Far away the sheet acts as a point mass k*Area/pi; at the centre of a
    large square it is the isotropic k*theta (Eq. alphapart with the sign of a
    positive sheet)."""
    rect = (-1.0, 2.0, -0.5, 0.5)
    k = 0.3
    mass = k * 3.0 * 1.0 / np.pi
    for t in [(3e3, 1e3), (-2e3, 4e3)]:
        o = np.array(oracle.sheet_positive(*rect, k, *t))
        c = np.array(t) - np.array([0.5, 0.0])  # centroid
        ref = mass * c / (c @ c)
        assert np.allclose(o, ref, rtol=1e-6)
    L = 200.0
    for t in [(0.3, -0.7), (1.2, 0.4)]:
        o = np.array(oracle.sheet_positive(-L, L, -L, L, k, *t))
        assert np.allclose(o, k * np.array(t), rtol=1e-4)


# --------------------------------------------------------- full deflection
def _field(params, plan, n, shape="equal", seed=1):
    box = (plan.a1, plan.a2, plan.b1, plan.b2)
    return lensgen.lens_field(n, box, shape=shape, seed=seed)


def test_deflection_divergence_is_kappa_s():
    """Eq. (alpha1): away from lenses the lens sum is divergence free, the
    matrix term gives 2 kappa and the NEGATIVE sheet -2 kappa_*, so
    div(alpha) = 2 kappa_s.  Catches a positive sheet (the appendix's sign taken as is) or a matrix
    that forgets kappa_*."""
    p = oracle.make_params(0.35, 0.15, 0.4, (-1.0, 1.0, -1.0, 1.0), 16, 4.0)
    q = oracle.size(p)
    xy, m = _field(p, q, 40, "uniform", seed=7)
    h = 1e-5
    rng = np.random.default_rng(3)
    for _ in range(6):
        x = rng.uniform(q.a1 + 1, q.a2 - 1)
        y = rng.uniform(q.b1 + 1, q.b2 - 1)
        if np.min(np.hypot(xy[:, 0] - x, xy[:, 1] - y)) < 0.05:
            continue
        f = lambda a, b: np.array(oracle.deflection(p, q, xy, m, a, b))
        dx = (f(x + h, y) - f(x - h, y)) / (2 * h)
        dy = (f(x, y + h) - f(x, y - h)) / (2 * h)
        assert abs(dx[0] + dy[1] - 2 * p.kappa_s) < 1e-4
        # shear from the matrix is +gamma in alpha_1 / theta_1 minus alpha_2 / theta_2
        assert abs(dx[1] - dy[0]) < 1e-4


def test_deflection_circle_plane_matches_eq_alpha():
    """Eq. (alpha) for the circular plane centred on the origin: the smooth
    part is diag(k_s + g, k_s - g) theta, no sheet, no kappa_* in the matrix."""
    p = oracle.make_params(0.3, 0.1, 0.2, (-1.0, 1.0, -1.0, 1.0), 8, 4.0,
                           plane=oracle.PLANE_CIRCLE)
    q = oracle.size(p)
    assert abs(q.cx) < 1e-15 and abs(q.cy) < 1e-15
    xy = np.array([[0.5, -0.25], [-1.0, 2.0]])
    m = np.array([1.0, 0.5])
    t = np.array([0.7, 0.3])
    d = t - xy
    ref = np.array([(0.1 + 0.2) * t[0], (0.1 - 0.2) * t[1]]) + (m[:, None] * d /
                                                              (d * d).sum(1)[:, None]).sum(0)
    assert np.allclose(oracle.deflection(p, q, xy, m, *t), ref, rtol=0, atol=1e-14)


def _disc_sheet_quadrature(cx, cy, R, k, t1, t2, npts=4096):
    """Deflection of a POSITIVE uniform disc of density k, radius R, centre
    (cx, cy), at a point inside it, by an independent route: in polar
    coordinates about the field point the 2-D integral
    (k/pi) int (theta - theta') / |theta - theta'|^2 d^2 theta' reduces to
    -(k/pi) int_0^2pi rho(phi) u(phi) dphi, with u = (cos phi, sin phi) and
    rho(phi) the distance to the disc's edge along u; the integrand is smooth
    and periodic, so the trapezoid rule converges geometrically."""
    phi = np.arange(npts) * (2.0 * np.pi / npts)
    ux, uy = np.cos(phi), np.sin(phi)
    px, py = t1 - cx, t2 - cy
    pu = px * ux + py * uy
    rho = -pu + np.sqrt(pu * pu - (px * px + py * py) + R * R)
    w = 2.0 * np.pi / npts
    return (-(k / np.pi) * w * np.sum(rho * ux), -(k / np.pi) * w * np.sum(rho * uy))


def test_disc_quadrature_route_is_newtons_theorem():
    """The quadrature helper itself: a centred point sees no pull, and inside
    an off-centre disc the pull is k (theta - theta_c) (Newton's theorem, the
    circle limit of Eq. (alphapart) with the sign of a positive sheet)."""
    assert np.allclose(_disc_sheet_quadrature(1.0, -2.0, 3.0, 0.4, 1.0, -2.0), (0.0, 0.0), atol=1e-14)
    for t in [(2.5, -1.0), (-1.2, -3.9), (1.0, 0.9)]:
        o = _disc_sheet_quadrature(1.0, -2.0, 3.0, 0.4, *t)
        assert np.allclose(o, (0.4 * (t[0] - 1.0), 0.4 * (t[1] + 2.0)), rtol=0, atol=1e-12)


@pytest.mark.parametrize("src", [(1.0, 3.0, -2.5, -0.5), (-7.0, -3.0, 4.0, 9.0)])
def test_off_centre_circle_plane_is_eq_alpha1_with_the_disc_sheet(src):
    """Eq. (alpha1) with the circular negative sheet of a plane NOT centred on
    the origin: the matrix term diag(k + g, k - g) theta with k = k_s + k_*
    (k_* of the lenses passed in), the lens sum, and minus the disc's own pull
    computed by quadrature (not by the oracle's k_* theta_c closed form).
    Catches a dropped or sign-flipped k_* theta_c term of the oracle's circle
    branch, or a disc centred on the origin instead of the plane centre."""
    p = oracle.make_params(0.3, 0.1, 0.2, src, 16, 4.0, plane=oracle.PLANE_CIRCLE)
    q = oracle.size(p)
    assert np.hypot(q.cx, q.cy) > 2.0  # theta_c far from the origin
    xy, m = lensgen.lens_field(60, None, shape="uniform", seed=13, disc=(q.cx, q.cy, q.circle_r))
    ks = m.sum() / q.circle_r ** 2  # pi sum(m) / (pi R^2)
    kap = p.kappa_s + ks
    rng = np.random.default_rng(8)
    for _ in range(5):
        t = np.array([rng.uniform(q.a1, q.a2), rng.uniform(q.b1, q.b2)])
        d = t - xy
        lens = (m[:, None] * d / (d * d).sum(1)[:, None]).sum(0)
        disc = np.array(_disc_sheet_quadrature(q.cx, q.cy, q.circle_r, ks, *t))
        ref = np.array([(kap + p.gamma) * t[0], (kap - p.gamma) * t[1]]) + lens - disc
        assert np.allclose(oracle.deflection(p, q, xy, m, *t), ref, rtol=0, atol=1e-10)


@pytest.mark.parametrize("plane", [oracle.PLANE_RECT, oracle.PLANE_CIRCLE])
def test_translation_covariance_of_the_lens_equation(plane):
    """Moving the source region by d_beta moves the plane centre by
    theta_c = (d_beta_1 / (1 - k - g), d_beta_2 / (1 - k + g)); with every lens
    moved by theta_c too, each lattice ray must land exactly d_beta away
    (beta' - beta = diag(1 - k - g, 1 - k + g) theta_c with the sheet moving
    with the plane), so the two maps agree pixel for pixel.  A missing or
    sign-flipped k_* theta_c term (circle) or a sheet that does not follow the
    plane (rectangle) shifts every ray by k_* theta_c instead."""
    base = (-2.5, 2.5, -2.5, 2.5)
    dbeta = (3.25, -1.75)
    moved = (base[0] + dbeta[0], base[1] + dbeta[0], base[2] + dbeta[1], base[3] + dbeta[1])
    args = (0.3, 0.05, 0.25)
    p0 = oracle.make_params(*args, base, 24, 9.3, plane=plane)
    p1 = oracle.make_params(*args, moved, 24, 9.3, plane=plane)
    q0, q1 = oracle.size(p0), oracle.size(p1)
    assert (q0.nrx, q0.nry) == (q1.nrx, q1.nry)
    tc = np.array([q1.cx - q0.cx, q1.cy - q0.cy])
    lam = np.array([1.0 - q0.kappa - p0.gamma, 1.0 - q0.kappa + p0.gamma])
    assert np.allclose(lam * tc, dbeta, rtol=1e-14, atol=1e-14)
    if plane == oracle.PLANE_CIRCLE:
        xy0, m = lensgen.lens_field(80, None, shape="uniform", seed=21, disc=(q0.cx, q0.cy, q0.circle_r))
    else:
        xy0, m = lensgen.lens_field(80, (q0.a1, q0.a2, q0.b1, q0.b2), shape="uniform", seed=21)
    m = m * (0.3 / oracle.kappa_star_actual(p0, q0, m))  # kappa_* = 0.3 exactly
    xy1 = xy0 + tc
    idx = np.random.default_rng(4).integers(0, q0.n_rays, 400)
    _, b0, _ = oracle.shoot_rays(p0, q0, xy0, m, idx)
    _, b1, _ = oracle.shoot_rays(p1, q1, xy1, m, idx)
    assert np.allclose(b1 - b0, dbeta, rtol=0, atol=1e-9)
    c0, _, n0 = oracle.make_map(p0, q0, xy0, m)
    c1, _, n1 = oracle.make_map(p1, q1, xy1, m)
    # rays within rounding of a pixel edge may go either way
    assert np.abs(c0.astype(np.int64) - c1.astype(np.int64)).sum() <= 4
    assert abs(n0 - n1) <= 2 and n0 > 1000


def test_tiny_field_against_quadrature_route():
    """Brute force on a tiny input by an independent route: numpy lens sum plus
    the rectangle sheet by 2-D quadrature (not the closed form)."""
    p = oracle.make_params(0.2, 0.05, 0.1, (-0.5, 0.5, -0.5, 0.5), 4, 1.0, border=0.5)
    q = oracle.size(p)
    xy, m = _field(p, q, 3, "uniform", seed=11)
    ks = np.pi * m.sum() / (q.ix * q.iy)
    rng = np.random.default_rng(5)
    for _ in range(3):
        t = np.array([rng.uniform(q.a1, q.a2), rng.uniform(q.b1, q.b2)])
        d = t - xy
        lens = (m[:, None] * d / (d * d).sum(1)[:, None]).sum(0)
        sheet = np.array(_quad_sheet(q.a1, q.a2, q.b1, q.b2, ks, *t))
        kap = p.kappa_s + ks
        ref = np.array([(kap + p.gamma) * t[0], (kap - p.gamma) * t[1]]) + lens - sheet
        assert np.allclose(oracle.deflection(p, q, xy, m, *t), ref, rtol=0, atol=1e-10)


# ------------------------------------------------------------- maps
def _paczynski_pixel_mean(x0, y0, s, order=16):
    g, w = leggauss(order)
    X = x0 + (g + 1) / 2 * s
    Y = y0 + (g + 1) / 2 * s
    XX, YY = np.meshgrid(X, Y)
    u = np.hypot(XX, YY)
    mu = (u * u + 2) / (u * np.sqrt(u * u + 4))
    return np.einsum("i,j,ij->", w, w, mu) / 4


def test_point_lens_paczynski():
    """One unit lens at the origin, circular plane, no smooth matter or shear:
    every pixel's magnification is the pixel average of Paczynski's
    mu(u) = (u^2+2)/(u sqrt(u^2+4)).  A regular ray lattice converges like
    N^(-3/4) (Sec. 3.2), so each pixel must sit within 3 N^(-3/4)."""
    n = 40
    p = oracle.make_params(0.0, 0.0, 0.0, (-2.0, 2.0, -2.0, 2.0), n, 2500.0, border=1.5,
                           plane=oracle.PLANE_CIRCLE)
    q = oracle.size(p)
    counts, mag, landed = oracle.make_map(p, q, np.zeros((1, 2)), np.ones(1))
    assert counts.sum() == landed
    s = q.sx
    worst, sq = 0.0, []
    for iy in range(n):
        for ix in range(n):
            x0, y0 = -2 + ix * s, -2 + iy * s
            umin = np.hypot(np.clip(0, x0, x0 + s), np.clip(0, y0, y0 + s))
            if umin < 0.1:
                continue
            ex = _paczynski_pixel_mean(x0, y0, s)
            rel = (mag[iy, ix] - ex) / ex
            nexp = ex * p.rays_per_pixel
            worst = max(worst, abs(rel) * nexp ** 0.75)
            sq.append(rel * rel)
    assert worst < 3.0
    assert np.sqrt(np.mean(sq)) < 2e-3


@pytest.mark.parametrize("ks,kstar,g", [(0.2, 0.0, 0.1), (0.2, 0.3, 0.1), (1.3, 0.0, -0.25)])
def test_lens_free_sheet_counts(ks, kstar, g):
    """No lenses: the map is the linear smooth mapping diag(1-k-g, 1-k+g) of a
    regular lattice (Eq. lensequation with N_* = 0; declared kappa_* without
    lenses adds nothing: the sheet uses the density of the lenses passed in).  Each pixel holds between
    floor(wx)floor(wy) and ceil(wx)ceil(wy) rays, w = s / (|lambda| dx3), and
    the mean magnification is 1/|(1-k)^2 - g^2|."""
    p = oracle.make_params(kstar, ks, g, (-1.0, 1.5, -1.2, 0.8), (24, 16), 37.0)
    q = oracle.size(p)
    counts, mag, landed = oracle.make_map(p, q, np.zeros((0, 2)), np.zeros(0))
    l1, l2 = 1 - ks - g, 1 - ks + g
    wx, wy = q.sx / (abs(l1) * q.dx3), q.sy / (abs(l2) * q.dx3)
    assert counts.min() >= np.floor(wx) * np.floor(wy)
    assert counts.max() <= np.ceil(wx) * np.ceil(wy)
    mu0 = 1.0 / abs(l1 * l2)
    assert abs(mag.mean() / mu0 - 1) < 3.0 / min(wx, wy)
    assert counts.sum() == landed


def test_ray_conservation_and_chunk_additivity():
    """Integer invariants: counts sum to the landed rays, landed <= shot, and
    maps of disjoint lattice bands add up to the full map."""
    p = oracle.make_params(0.3, 0.0, 0.3, (-2.5, 2.5, -2.5, 2.5), 32, 4.0)
    q = oracle.size(p)
    xy, m = _field(p, q, 61, seed=1)
    full, _, landed = oracle.make_map(p, q, xy, m)
    assert full.sum() == landed <= q.n_rays
    mid = q.nry // 3
    c1, _, l1 = oracle.make_map(p, q, xy, m, rows=(0, mid))
    c2, _, l2 = oracle.make_map(p, q, xy, m, rows=(mid, q.nry))
    assert np.array_equal(c1 + c2, full) and l1 + l2 == landed


def test_mean_magnification():
    """Averaged over lens fields the map's mean magnification is the smooth
    1/|(1-kappa)^2 - gamma^2|.  The protective border (10 sqrt(kappa_*), flow
    chart) keeps the loss of rays below 2 % (Sec. 2.3), so the mean over 40
    seeded fields sits within that loss and three standard errors."""
    S = 16.0
    p = oracle.make_params(0.3, 0.1, 0.2, (-S / 2, S / 2, -S / 2, S / 2), 16, 16.0)
    q = oracle.size(p)
    n = int(round(q.n_star_paper))
    means = []
    for seed in range(40):
        xy, m = _field(p, q, n, seed=100 + seed)
        _, mag, _ = oracle.make_map(p, q, xy, m)
        means.append(mag.mean())
    mu0 = 1.0 / abs((1 - q.kappa) ** 2 - p.gamma ** 2)
    rel = np.mean(means) / mu0 - 1
    sem = np.std(means) / mu0 / np.sqrt(len(means))
    assert -0.02 - 3 * sem < rel < 3 * sem


def test_paper_lens_count():
    """Sizing against a printed number: fig:Performance's field (kappa = gamma
    = 0.3, f_* = 1, S = 20 theta_E) holds N_* = 238 lenses of mean mass 1."""
    g = json.load(open(os.path.join(GOLDEN, "fig_performance_nstar.json")))
    k = g["kappa"]
    p = oracle.make_params(k * g["f_star"], k * (1 - g["f_star"]), g["gamma"],
                           (-g["S_scale"] / 2, g["S_scale"] / 2, -g["S_scale"] / 2,
                            g["S_scale"] / 2), 1024, 10.0)
    q = oracle.size(p)
    assert abs(q.border - 10 * np.sqrt(0.3)) < 1e-12
    assert abs(q.n_star_paper / g["N_star_printed"] - 1) < 0.06


def test_sizing_flow_chart():
    """Flow-chart sizing: P = 10 sqrt(kappa_*), I = (S + 2P)/|1 - kappa -+ gamma|,
    widened to a whole number of rays of side sqrt(s^2 / N_av), N_av per unlensed source pixel,
    centred on the image of the source centre."""
    p = oracle.make_params(0.45, 0.0, 0.45, (-10.0, 10.0, -10.0, 10.0), 2000, 100.0)
    q = oracle.size(p)
    P = 10 * np.sqrt(0.45)
    assert abs(q.ix0 - (20 + 2 * P) / 0.1) < 1e-9 and abs(q.iy0 - (20 + 2 * P) / 1.0) < 1e-9
    assert abs(q.dx3 - 0.001) < 1e-15
    assert q.ix0 <= q.ix < q.ix0 + q.dx3 and q.iy0 <= q.iy < q.iy0 + q.dx3
    assert abs(q.a1 + q.a2) < 1e-9 and abs(q.b1 + q.b2) < 1e-9
    with pytest.raises(ValueError):
        oracle.size(oracle.make_params(0.5, 0.0, 0.5, (-1, 1, -1, 1), 8, 4.0))
