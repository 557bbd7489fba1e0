"""Direct pins of the oracle's small helpers (each also used inside the larger pinned
quantities): the contour of Eq. 8, the pair geometry and rotation classes of the fill,
the slab wavenumber, the alpha node count, sinc and the Gaussian transform.  Every
check is fixed by a closed form, an identity or an independent computation."""
import math

import numpy as np

from oracle import contour as oc, fill as of, green as og, reaction as orx, spectra as osp


def test_parabola_peak_ends_and_symmetry():
    bp, hgt = 12.0, 0.05
    assert abs(oc.beta_imag(bp / 2, bp, hgt) - hgt) < 1e-15          # peak height H at beta_p / 2
    assert oc.beta_imag(0.0, bp, hgt) == 0.0 and oc.beta_imag(bp, bp, hgt) == 0.0
    assert oc.beta_imag(1.5 * bp, bp, hgt) == 0.0                     # real axis beyond beta_p
    b = np.linspace(0.1, bp - 0.1, 7)
    assert np.allclose(oc.beta_imag(b, bp, hgt), oc.beta_imag(bp - b, bp, hgt), rtol=0, atol=1e-15)


def test_slope_is_the_derivative():
    bp, hgt = 12.0, 0.05
    b = np.linspace(0.3, bp - 0.3, 9)
    d = 1e-6
    fd = (oc.beta_imag(b + d, bp, hgt) - oc.beta_imag(b - d, bp, hgt)) / (2 * d)
    assert np.allclose(oc.beta_imag_slope(b, bp, hgt), fd, rtol=0, atol=1e-9)
    # the paper's ratio gamma = beta_I / beta_R at beta_R -> 0 is the slope there, 4 H / beta_p
    assert abs(oc.beta_imag_slope(0.0, bp, hgt) - 4 * hgt / bp) < 1e-15
    assert oc.beta_imag_slope(bp + 1.0, bp, hgt) == 0.0


def test_contour_weights_integrate_the_measure_exactly():
    """sum_j w_j = int_C d beta_c = beta_c(beta_max) - beta_c(0) = beta_max: the midpoint
    rule is exact for the linear slope when beta_p sits on a cell boundary."""
    n, bmax = 1000, 40.0
    h = bmax / n
    bp = 337 * h
    nd = oc.contour_nodes(n, bmax, bp, 0.07)
    assert abs(nd["weight"].sum() - bmax) < 1e-12 * bmax
    assert np.allclose(nd["beta_r"], (np.arange(n) + 0.5) * h)
    bc, dbc = oc.contour_point(nd["beta_r"], bp, 0.07)
    assert np.allclose(bc, nd["beta_c"]) and np.allclose(dbc * h, nd["weight"])


def test_rectangle_rule_on_the_contour_is_second_order():
    """int_C exp(i a beta) d beta = (exp(i a beta_max) - 1) / (i a) (Cauchy: any contour
    from 0 to beta_max); the midpoint rule on the nodes converges at order 2."""
    a, bmax = 0.7, 30.0
    exact = (np.exp(1j * a * bmax) - 1.0) / (1j * a)
    errs = []
    for n in (600, 1200, 2400):
        h = bmax / n
        nd = oc.contour_nodes(n, bmax, 120 * h * n / 600, 0.3)
        errs.append(abs(np.sum(nd["weight"] * np.exp(1j * a * nd["beta_c"])) - exact))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_pair_geometry_and_classes():
    pos = np.array([[1.0, 2.0], [4.0, 6.0]])
    rho, phi = of.pair_geometry(pos, 1, 0)        # Delta = r_1 - r_0 = (3, 4)
    assert rho == 5.0 and abs(phi - math.atan2(4.0, 3.0)) < 1e-15
    rho2, phi2 = of.pair_geometry(pos, 0, 1)      # the opposite pair: same rho, phi + pi
    assert rho2 == 5.0 and abs(math.remainder(phi2 - phi - math.pi, 2 * math.pi)) < 1e-15
    rot = np.array([0, 1])
    assert [of.class_index(rot, m, n) for m in (0, 1) for n in (0, 1)] == [0, 1, 2, 3]
    assert [tuple(orx.rotation_angles(c)) for c in range(4)] == [
        (0.0, 0.0), (0.0, math.pi / 2), (math.pi / 2, 0.0), (math.pi / 2, math.pi / 2)]


def test_slab_wavenumber():
    k0, eps = 2 * math.pi, 4.4
    b2 = np.array([0.5, 20.0, 40.0 + 0.3j, 200.0])
    k1 = og.kz_slab(b2, eps, k0)
    assert np.allclose(k1 * k1, eps * k0 ** 2 - b2, rtol=1e-14, atol=1e-12)
    assert np.all(k1.real >= 0.0)                 # principal root (k1 enters through even functions)


def test_alpha_node_count_resolves_the_integrand():
    for rho in (0.5, 5.0, 50.0):
        for q in (0, 16):
            npr = orx.alpha_nodes(rho, 66.0, q)
            assert 2 * npr > 66.0 * rho + q + 40
    assert orx.alpha_nodes(50.0, 66.0, 16) > orx.alpha_nodes(5.0, 66.0, 16)


def test_sinc_definition_series_and_complex_argument():
    assert osp.sinc(0.0) == 1.0
    z = np.array([0.999e-3, 1.001e-3, 0.3 + 0.2j, 2.0, -5.0j])
    direct = np.sin(z) / z
    assert np.allclose(osp.sinc(z), direct, rtol=1e-14, atol=0)   # both sides of the series switch
    y = 1.7
    assert abs(osp.sinc(1j * y) - math.sinh(y) / y) < 1e-15       # sin(iy)/(iy) = sinh(y)/y


def test_gaussian_transform_against_brute_force():
    """F(k) = int g(r) exp(-i k.r) dr for g = exp(-|r - c|^2 / (4 s^2)) / (4 pi s^2): a
    Riemann sum on a fine grid against the closed form exp(-s^2 k^2) exp(-i k.c)."""
    s, cx, cy = 0.3, 0.2, -0.1
    x = np.linspace(-4.0, 4.0, 801)
    X, Y = np.meshgrid(x, x, indexing="ij")
    dx = x[1] - x[0]
    g = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (4 * s * s)) / (4 * math.pi * s * s)
    for kx, ky in ((0.0, 0.0), (1.3, -0.4), (3.0, 2.0)):
        num = np.sum(g * np.exp(-1j * (kx * X + ky * Y))) * dx * dx
        assert abs(num - osp.gaussian_ft(kx, ky, cx, cy, s)) < 1e-10
