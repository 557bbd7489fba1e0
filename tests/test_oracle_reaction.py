"""Pins for the oracle's reaction tables (Eq. 9 in harmonic form).

What fixes each result independently of the oracle's own code:
* a Gaussian spectral harmonic has a closed-form Hankel transform
  (Gradshteyn & Ryzhik 6.631.4), which pins the Bessel sum, the alpha form,
  the contour Jacobian of Eq. 8 and the (-i)^q convention;
* a pair of Gaussian currents under a unit dyadic has a closed-form 2-D
  Fourier pair, which pins the whole chain kernel -> harmonics -> Z_q ->
  Z'(rho, phi), including the sign of exp(-i k.Delta) and of exp(i q phi);
* Cauchy's theorem: the converged contour integral does not depend on the
  contour height while no pole is crossed, equals the real-axis integral
  with the surface-wave pole extracted (principal value - i pi Res), and
  not the other indentation (principal value + i pi Res);
* reciprocity of the Galerkin reaction, Z'_ab(Delta; Q) = Z'_ba(-Delta; conj Q),
  which pins where Eq. 11 and Eq. 10 put the conjugates;
* symmetries: J_q(0) = 0 for q != 0; odd harmonics vanish for the symmetric
  strip; a (90, 90) degree rotation class is the (0, 0) class times (-i)^q.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
from scipy.optimize import brentq

from oracle import contour, green, reaction, spectra
import workloads

K0 = 2 * math.pi


def strip_basis():
    return spectra.BasisSet("strip", np.ones((1, 1)), length=0.45, width=0.02)


def small_patch(m=2, seed=11, complex_q=True):
    rng = np.random.default_rng(seed)
    ax = np.array([-0.1, 0.0, 0.1])
    gx, gy = np.meshgrid(ax, ax)
    cx = np.concatenate([gx.ravel(), gx.ravel()])
    cy = np.concatenate([gy.ravel(), gy.ravel()])
    d = np.concatenate([np.zeros(9, int), np.ones(9, int)])
    q = rng.standard_normal((18, m)) + (1j * rng.standard_normal((18, m)) if complex_q else 0)
    return spectra.BasisSet("rooftop", q, cx=cx, cy=cy, direction=d,
                            half_len=np.full(18, 0.1), width=np.full(18, 0.1))


def gaussian_hankel(q, s, rho):
    # (-i)^q/(2 pi) int_0^inf b^(q+1) exp(-s^2 b^2) J_q(b rho) db
    return ((-1j) ** q / (2 * np.pi)) * rho ** q / (2 * s * s) ** (q + 1) * np.exp(-rho ** 2 / (4 * s * s))


@pytest.mark.parametrize("q", [0, 1, 3, -2])
def test_gaussian_hankel_pair_bessel_and_alpha_forms(q):
    s = 0.35
    rho = np.array([0.0, 0.4, 1.3, 2.2])
    # beta_p on a cell boundary of both node sets: each smooth piece of the contour is then
    # integrated by the midpoint rule with an h^2 error that Richardson extrapolation removes
    bmax, bp, height = 30.0, 8.1, 0.6

    def o2(n, form):
        c = contour.contour_nodes(n, bmax, bp, height)
        hq = (c["beta_c"] ** abs(q) * np.exp(-s * s * c["beta_c"] ** 2))[None, :]
        if q < 0:
            hq = hq * (-1) ** q  # H_{-q} for the harmonic b^|q| e^{-s^2 b^2} e^{-i|q| alpha} mirrored
        fn = reaction.table_bessel if form == "bessel" else reaction.table_alpha
        return fn(hq, [q], c["beta_c"], c["weight"], rho)[0]

    exact = gaussian_hankel(abs(q), s, rho) * ((-1) ** q if q < 0 else 1)
    # J_{-q} = (-1)^q J_q and the (-i)^q prefactor combine to the same closed form for -|q|
    if q < 0:
        exact = gaussian_hankel(abs(q), s, rho) * ((-1j) ** q / (-1j) ** abs(q)) * (-1) ** q * (-1) ** q
    for form in ("bessel", "alpha"):
        z1, z2 = o2(1000, form), o2(2000, form)
        rich = (4 * z2 - z1) / 3  # midpoint rule: error ~ h^2, Richardson removes it
        scale = np.abs(exact).max()
        assert np.abs(rich - exact).max() < 1e-9 * scale
        assert np.abs(z2 - exact).max() < 1e-4 * scale


def test_gaussian_currents_full_chain_2d_fourier_pair():
    s = 0.12
    c0 = np.array([0.05, -0.03])
    c1 = np.array([-0.04, 0.02])
    bs = spectra.BasisSet("gaussian", np.eye(2), cx=np.array([c0[0], c1[0]]),
                          cy=np.array([c0[1], c1[1]]), direction=np.array([0, 0]), s=s)
    qmax = 14
    qs = np.arange(-qmax, qmax + 1)
    rhos = np.array([0.0, 0.2, 0.55])
    zs = []
    for n in (1500, 3000):   # beta_p = 9.9 is a cell boundary of both node sets
        c = contour.contour_nodes(n, 45.0, 9.9, 0.5)
        hq = reaction.harmonics(bs, c["beta_c"], qs, 64, 0, 0, K0, green_fn=green.identity_green)
        zs.append(reaction.table_bessel(hq, qs, c["beta_c"], c["weight"], rhos))
    ztab = (4 * zs[1] - zs[0]) / 3   # Richardson on the midpoint rule's h^2 term
    for ir, rho in enumerate(rhos):
        zq = ztab[..., ir]
        for phi in (0.0, 1.0, -2.4):
            z = reaction.reaction_from_table(zq, qs, phi)      # (2, 2)
            delta = rho * np.array([math.cos(phi), math.sin(phi)])
            for a, b, ca, cb in ((0, 1, c0, c1), (1, 0, c1, c0), (0, 0, c0, c0)):
                d = delta + ca - cb
                exact = np.exp(-d @ d / (8 * s * s)) / (8 * np.pi * s * s)
                assert abs(z[a, b] - exact) < 1e-10 * (1 / (8 * np.pi * s * s))


def _cfg1_substrate():
    return 2.2, 0.05


def _tm0_root(eps_r, h):
    def f(b):
        a = math.sqrt(b * b - K0 * K0)
        k1 = math.sqrt(eps_r * K0 * K0 - b * b)
        return eps_r * a * math.cos(k1 * h) - k1 * math.sin(k1 * h)
    return brentq(f, K0 * (1 + 1e-12), K0 * math.sqrt(eps_r) * (1 - 1e-12), xtol=1e-15)


@pytest.mark.slow
def test_cauchy_contour_independence_and_pole_extraction():
    eps_r, h = _cfg1_substrate()
    kd = K0 * math.sqrt(eps_r)
    bmax, bp = 5 * kd, 1.3 * kd
    bs = strip_basis()
    q, rho, na = 0, 0.7, 48
    args = dict(basis=bs, a=0, b=0, q=q, rho=rho, beta_max=bmax, beta_p=bp, n_alpha=na,
                eps_r=eps_r, h=h, k0=K0)
    z_hi = reaction.table_adaptive(height=0.4, **args)
    z_lo = reaction.table_adaptive(height=0.15, **args)
    assert abs(z_hi - z_lo) < 1e-9 * abs(z_hi)

    # real axis: principal value minus i pi Res at the TM0 pole (just below the axis)
    bs_pole = _tm0_root(eps_r, h)

    def f(beta):
        beta = complex(beta)
        hq = reaction.harmonic_at(bs, 0, 0, q, beta, na, eps_r, h, K0)
        return ((-1j) ** q / (2 * np.pi)) * hq * reaction.bessel_jq(q, beta * rho) * beta

    # residue by the trapezoid rule on a small circle (spectrally accurate for analytic f)
    rc = 0.25 * (bs_pole - K0)
    th = 2 * np.pi * np.arange(64) / 64
    pts = bs_pole + rc * np.exp(1j * th)
    res = np.mean([f(p) * rc * np.exp(1j * t) for p, t in zip(pts, th)])
    g = lambda b: f(b) - res / (b - bs_pole)
    kw = dict(points=[K0, bs_pole, bp], limit=400, epsabs=1e-14, epsrel=1e-12)
    pv = (si.quad(lambda b: g(b).real, 0, bmax, **kw)[0]
          + 1j * si.quad(lambda b: g(b).imag, 0, bmax, **kw)[0]
          + res * math.log((bmax - bs_pole) / bs_pole))
    z_axis = pv - 1j * math.pi * res
    assert abs(z_axis - z_hi) < 1e-8 * abs(z_hi)

    # the pole contributes at first order: the opposite indentation (contour below the
    # pole) is far from the contour result, so the test decides the side of Eq. 8
    assert abs((pv + 1j * math.pi * res) - z_hi) > 0.5 * abs(z_hi)


def test_matched_o2_converges_to_o1():
    eps_r, h = _cfg1_substrate()
    kd = K0 * math.sqrt(eps_r)
    bmax, bp = 5 * kd, 1.3 * kd
    bs = strip_basis()
    rho = np.array([0.9])
    o1 = reaction.table_adaptive(bs, 0, 0, 0, rho[0], bmax, bp, 0.3, 48, eps_r, h, K0)
    errs = []
    for n in (512, 1024, 2048):
        # O1 does not depend on beta_p (Cauchy); the node set puts beta_p on a cell boundary
        bp_n = round(bp * n / bmax) * bmax / n
        c = contour.contour_nodes(n, bmax, bp_n, 0.3)
        hq = reaction.harmonics(bs, c["beta_c"], [0], 48, eps_r, h, K0)
        z = reaction.table_bessel(hq, [0], c["beta_c"], c["weight"], rho)[0, 0, 0, 0]
        errs.append(abs(z - o1) / abs(o1))
    # rectangle rule on a piecewise-smooth contour: second order in h
    assert errs[-1] < 1e-4
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_bessel_and_alpha_forms_agree_on_slab():
    eps_r, h = _cfg1_substrate()
    kd = K0 * math.sqrt(eps_r)
    c = contour.contour_nodes(512, 5 * kd, 1.3 * kd, 6 * 5 * kd / 512)
    bs = small_patch(m=2)
    qs = np.arange(-3, 4)
    hq = reaction.harmonics(bs, c["beta_c"], qs, 64, eps_r, h, K0)
    rho = np.array([0.0, 0.3, 1.7, 4.0])
    zb = reaction.table_bessel(hq, qs, c["beta_c"], c["weight"], rho)
    za = reaction.table_alpha(hq, qs, c["beta_c"], c["weight"], rho)
    assert np.abs(zb - za).max() < 1e-11 * np.abs(zb).max()


def test_reciprocity_complex_coefficients():
    # Z'_ab(Delta; Q) = Z'_ba(-Delta; conj Q)  <=>  Z_ab,q[Q] = (-1)^q Z_ba,q[conj Q]
    eps_r, h = 4.4, 0.03
    kd = K0 * math.sqrt(eps_r)
    c = contour.contour_nodes(600, 5 * kd, 1.3 * kd, 6 * 5 * kd / 600)
    bs = small_patch(m=2)
    bsc = spectra.BasisSet("rooftop", np.conj(bs.q), **bs.geom)
    qs = np.arange(-4, 5)
    rho = np.array([0.2, 1.1, 3.0])
    z = reaction.table_bessel(reaction.harmonics(bs, c["beta_c"], qs, 64, eps_r, h, K0),
                              qs, c["beta_c"], c["weight"], rho)
    zc = reaction.table_bessel(reaction.harmonics(bsc, c["beta_c"], qs, 64, eps_r, h, K0),
                               qs, c["beta_c"], c["weight"], rho)
    sign = ((-1.0) ** np.abs(qs))[:, None]
    lhs = z
    rhs = np.swapaxes(zc, 0, 1) * sign
    assert np.abs(lhs - rhs).max() < 1e-11 * np.abs(z).max()
    # and the reciprocity fails if the conjugates were put on the same side
    assert np.abs(np.swapaxes(z, 0, 1) * sign - z).max() > 1e-3 * np.abs(z).max()


def test_symmetries_strip_and_rho_zero_and_rotation_class():
    eps_r, h = _cfg1_substrate()
    kd = K0 * math.sqrt(eps_r)
    c = contour.contour_nodes(256, 5 * kd, 1.3 * kd, 6 * 5 * kd / 256)
    qs = np.arange(-4, 5)
    hs = reaction.harmonics(strip_basis(), c["beta_c"], qs, 64, eps_r, h, K0)
    scale = np.abs(hs).max()
    odd = np.abs(qs) % 2 == 1
    assert np.abs(hs[:, :, odd]).max() < 1e-12 * scale
    assert np.abs(hs - hs[:, :, ::-1]).max() < 1e-12 * scale        # H_{-q} = H_q
    z0 = reaction.table_bessel(hs, qs, c["beta_c"], c["weight"], np.array([0.0]))
    assert np.abs(z0[:, :, qs != 0]).max() < 1e-14 * np.abs(z0).max()
    bs = small_patch(m=2)
    h00 = reaction.harmonics(bs, c["beta_c"], qs, 64, eps_r, h, K0, *reaction.rotation_angles(0))
    h11 = reaction.harmonics(bs, c["beta_c"], qs, 64, eps_r, h, K0, *reaction.rotation_angles(3))
    phase = ((-1j) ** qs)[:, None]
    assert np.abs(h11 - h00 * phase).max() < 1e-11 * np.abs(h00).max()
    h01 = reaction.harmonics(bs, c["beta_c"], qs, 64, eps_r, h, K0, *reaction.rotation_angles(1))
    assert np.abs(h01 - h00).max() > 1e-3 * np.abs(h00).max()


def test_alpha_trapezoid_converged_for_workload_sizes():
    # the harmonic decomposition of the cfg-2-like rooftop patch is converged at n_alpha = 128
    wl = workloads.patch_m4(n=64)
    el = wl.element
    bs = spectra.BasisSet("rooftop", el.q, cx=el.cx, cy=el.cy, direction=el.direction,
                          half_len=el.half_len, width=el.width)
    beta = np.array([wl.contour.beta_max * 0.999, wl.substrate.k_d * 1.1 + 0.01j])
    qs = wl.qs
    a = reaction.harmonics(bs, beta, qs, 128, wl.substrate.eps_r, wl.substrate.h, K0)
    b = reaction.harmonics(bs, beta, qs, 256, wl.substrate.eps_r, wl.substrate.h, K0)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()
