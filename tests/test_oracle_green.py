"""Pins for the oracle's grounded-slab Green's function.

The paper does not print G~ (it cites it); these tests tie the oracle's formula
to physics that is fixed independently of it: the textbook surface-wave
dispersion relations of a grounded slab, the thin-slab static limit,
rotational covariance of a dyadic in a horizontally isotropic medium, the
radiation condition on the free-space branch, and the side of the real axis
on which lossy-substrate poles lie (which decides the side of the contour of
Eq. 8).
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import green

K0 = 2 * math.pi


def tm_textbook(beta, eps_r, h, k0=K0):
    """TM surface waves of a grounded slab: eps_r * a = k1 tan(k1 h), a = sqrt(beta^2 - k0^2)."""
    a = math.sqrt(beta ** 2 - k0 ** 2)
    k1 = math.sqrt(eps_r * k0 ** 2 - beta ** 2)
    return eps_r * a * math.cos(k1 * h) - k1 * math.sin(k1 * h)


def te_textbook(beta, eps_r, h, k0=K0):
    """TE surface waves of a grounded slab: -k1 cot(k1 h) = a."""
    a = math.sqrt(beta ** 2 - k0 ** 2)
    k1 = math.sqrt(eps_r * k0 ** 2 - beta ** 2)
    return k1 * math.cos(k1 * h) + a * math.sin(k1 * h)


def _scale(beta, eps_r, h):
    te, tm = green.te_tm(beta ** 2, eps_r, h, K0)
    return abs(tm), abs(te)


@pytest.mark.parametrize("eps_r,h,expect", [(2.2, 0.05, 1.0150), (4.4, 0.03, 1.0113)])
def test_tm0_pole_is_zero_of_tm(eps_r, h, expect):
    kd = K0 * math.sqrt(eps_r)
    root = brentq(lambda b: tm_textbook(b, eps_r, h), K0 * (1 + 1e-12), kd * (1 - 1e-12),
                  xtol=1e-15)
    assert abs(root / K0 - expect) < 5e-4
    te, tm = green.te_tm(np.array(root ** 2), eps_r, h, K0)
    # Tm vanishes at the textbook root (relative to its size nearby), Te does not.
    te_n, tm_n = green.te_tm(np.array((root * 1.01) ** 2), eps_r, h, K0)
    assert abs(tm) < 1e-10 * abs(tm_n)
    assert abs(te) > 1e-3 * abs(te_n)


def test_te1_pole_thick_high_permittivity_slab():
    eps_r, h = 10.0, 0.1
    kd = K0 * math.sqrt(eps_r)
    grid = np.linspace(K0 * (1 + 1e-9), kd * (1 - 1e-9), 20001)
    vals = np.array([te_textbook(b, eps_r, h) for b in grid])
    idx = np.nonzero(np.sign(vals[:-1]) != np.sign(vals[1:]))[0]
    assert idx.size >= 1
    root = brentq(lambda b: te_textbook(b, eps_r, h), grid[idx[0]], grid[idx[0] + 1], xtol=1e-15)
    te, _ = green.te_tm(np.array(root ** 2), eps_r, h, K0)
    te_n, _ = green.te_tm(np.array((root * 1.01) ** 2), eps_r, h, K0)
    assert abs(te) < 1e-9 * abs(te_n)


def test_free_space_branch_radiation_condition():
    # propagating: k2 real positive; evanescent: k2 = -j sqrt(beta^2 - k0^2)
    b = np.array([0.3, 0.9]) * K0
    k2 = green.kz_free(b ** 2, K0)
    assert np.allclose(k2, np.sqrt(K0 ** 2 - b ** 2), rtol=1e-14)
    b = np.array([1.1, 3.0]) * K0
    k2 = green.kz_free(b ** 2, K0)
    assert np.allclose(k2, -1j * np.sqrt(b ** 2 - K0 ** 2), rtol=1e-14)
    # upper half of the beta plane (the contour side): Im k2 < 0
    bc = np.array([0.5, 1.0, 1.5]) * K0 + 0.05j
    assert np.all(green.kz_free(bc ** 2, K0).imag < 0)


def test_thin_slab_static_limit():
    # h -> 0: G ~ -j Z0 k0 h I + j Z0 h k k^T / (eps_r k0)   (current sheet over ground)
    eps_r = 3.0
    kx = np.array([0.3, 1.7, 4.0]) * K0
    ky = np.array([0.8, -0.4, 2.5]) * K0
    errs = []
    for h in (1e-4, 1e-5, 1e-6):
        gxx, gxy, gyy = green.dyadic_green(kx, ky, eps_r, h, K0)
        exx = -1j * green.Z0 * K0 * h + 1j * green.Z0 * h * kx * kx / (eps_r * K0)
        eyy = -1j * green.Z0 * K0 * h + 1j * green.Z0 * h * ky * ky / (eps_r * K0)
        exy = 1j * green.Z0 * h * kx * ky / (eps_r * K0)
        scale = np.abs(exx) + np.abs(eyy)
        errs.append(max(np.max(np.abs(gxx - exx) / scale), np.max(np.abs(gyy - eyy) / scale),
                        np.max(np.abs(gxy - exy) / scale)))
    # the relative deviation is first order in k0 h: it shrinks tenfold per decade of h
    assert errs[-1] < 1e-5
    assert 9.0 < errs[0] / errs[1] < 11.0 and 9.0 < errs[1] / errs[2] < 11.0


def test_rotational_covariance():
    # G(R k) = R G(k) R^T for any rotation (isotropic in the transverse plane); pins the
    # sign and size of the off-diagonal term relative to the diagonal ones.
    eps_r, h = 4.4, 0.03
    k = np.array([1.3 * K0 + 0.02j, 0.7 * K0 + 0.01j])
    for th in (0.3, 1.1, 2.5):
        r = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        rk = r @ k
        gxx, gxy, gyy = green.dyadic_green(k[0], k[1], eps_r, h, K0)
        g = np.array([[gxx, gxy], [gxy, gyy]])
        gxx2, gxy2, gyy2 = green.dyadic_green(rk[0], rk[1], eps_r, h, K0)
        g2 = np.array([[gxx2, gxy2], [gxy2, gyy2]])
        assert np.allclose(g2, r @ g @ r.T, rtol=1e-12, atol=1e-12 * np.abs(g).max())


def test_lossy_pole_below_real_axis():
    # With exp(+j w t) a lossy slab, eps_r (1 - j tan d), moves the TM0 pole below the real
    # axis; the lossless limit of the real-axis integral therefore passes ABOVE the pole,
    # which is the side the contour of Eq. 8 takes (beta_I >= 0).
    eps_r, h = 2.2, 0.05
    b = brentq(lambda x: tm_textbook(x, eps_r, h), K0 * (1 + 1e-12), K0 * math.sqrt(eps_r) * (1 - 1e-12))
    eps_l = eps_r * (1 - 0.01j)
    z = complex(b)
    for _ in range(60):  # Newton on Tm(beta) with a complex-step-free finite difference
        f = green.te_tm(np.array(z * z), eps_l, h, K0)[1]
        d = 1e-7
        fp = (green.te_tm(np.array((z + d) ** 2), eps_l, h, K0)[1] - f) / d
        z = z - complex(f / fp)
    assert abs(complex(green.te_tm(np.array(z * z), eps_l, h, K0)[1])) < 1e-9
    assert z.imag < 0


def test_vanishing_slab_gives_zero():
    kx = np.array([0.5, 2.0]) * K0
    ky = np.array([0.1, 1.0]) * K0
    g = green.dyadic_green(kx, ky, 2.2, 0.0, K0)
    assert all(np.all(np.abs(c) == 0) for c in g)


def tl_dyadic(kx, ky, eps_r, h, k0, z0):
    """The same dyadic from the transverse-resonance (transmission-line) picture, derived
    independently of the oracle's closed form: along k the current sees the TM line, across
    k the TE line, each an air half-space (admittance k2/(w mu0) for TE, w eps0/k2 for TM)
    in parallel with the slab line shorted by the ground plane at depth h
    (-j cot(k1 h) times k1/(w mu0), resp. w eps0 eps_r/k1).  With E = -Z J along each
    direction, G = -Z_TE I - (Z_TM - Z_TE) k k^T / beta^2."""
    kx = np.asarray(kx, dtype=np.complex128)
    ky = np.asarray(ky, dtype=np.complex128)
    b2 = kx * kx + ky * ky
    k2 = -1j * np.sqrt(b2 - k0 * k0 + 0j)            # Im k2 <= 0 (radiation condition)
    k1 = np.sqrt(eps_r * k0 * k0 - b2 + 0j)
    w_mu0, w_eps0 = k0 * z0, k0 / z0
    cot = np.cos(k1 * h) / np.sin(k1 * h)
    z_te = 1.0 / (k2 / w_mu0 - 1j * k1 * cot / w_mu0)
    z_tm = 1.0 / (w_eps0 / k2 - 1j * w_eps0 * eps_r * cot / k1)
    gxx = -z_te - (z_tm - z_te) * kx * kx / b2
    gxy = -(z_tm - z_te) * kx * ky / b2
    gyy = -z_te - (z_tm - z_te) * ky * ky / b2
    return gxx, gxy, gyy


@pytest.mark.parametrize("eps_r,h", [(2.2, 0.05), (4.4, 0.03), (10.0, 0.1)])
def test_dyadic_matches_transmission_line_model(eps_r, h):
    """Every order of the numerators (not only the leading thin-slab terms) against the
    transmission-line derivation, on the real axis below and above k0 and on the contour
    side of the plane (beta_I > 0), including points next to the surface-wave poles."""
    kd = K0 * math.sqrt(eps_r)
    betas = np.array([0.37 * K0, 0.99 * K0, 1.02 * K0, 0.5 * (K0 + kd), 0.98 * kd, 1.7 * kd, 4.6 * kd])
    betas = np.concatenate([betas, betas + 0.03j, betas[2:] + 0.2j])
    alphas = np.linspace(0.1, 2.9, betas.size)
    kx, ky = betas * np.cos(alphas), betas * np.sin(alphas)
    got = green.dyadic_green(kx, ky, eps_r, h, K0)
    ref = tl_dyadic(kx, ky, eps_r, h, K0, green.Z0)
    scale = np.maximum(np.abs(ref[0]), np.abs(ref[2]))
    for g, r in zip(got, ref):
        assert np.all(np.abs(g - r) <= 1e-11 * scale)


def test_remainder_vanishes_for_an_air_slab():
    """With eps_r = 1 the grounded slab is free space above a ground plane, which is exactly
    the extracted homogeneous medium (eps_eff = 1) and its image: Z^l's Green's function is
    zero at real and complex beta, in every component."""
    from oracle import green as og
    k0 = 2 * np.pi
    rem = og.layered_remainder()
    for b in (0.3, 1.5, 3.0, 6.5, 10.0, 40.0):
        for bi in (0.0, 0.2):
            kx, ky = (b + 1j * bi) * 0.6, (b + 1j * bi) * 0.8
            full = og.dyadic_green(kx, ky, 1.0, 0.05, k0)
            part = rem(kx, ky, 1.0, 0.05, k0)
            scale = max(abs(full[0]), abs(full[1]), abs(full[2]))
            assert max(abs(part[0]), abs(part[1]), abs(part[2])) < 1e-13 * scale


def test_remainder_loses_the_growing_charge_term():
    """On a dielectric slab the full dyadic grows like beta at large beta (the charge term),
    the remainder after extracting the eps_eff = (eps_r + 1)/2 medium and its image falls
    off; a flipped image sign breaks the air-slab identity."""
    from oracle import green as og
    k0 = 2 * np.pi
    rem = og.layered_remainder()
    g100 = og.dyadic_green(60.0, 80.0, 4.4, 0.03, k0)
    g400 = og.dyadic_green(240.0, 320.0, 4.4, 0.03, k0)
    r100 = rem(60.0, 80.0, 4.4, 0.03, k0)
    r400 = rem(240.0, 320.0, 4.4, 0.03, k0)
    for c in range(3):
        assert abs(g400[c]) / abs(g100[c]) > 3.0
        assert abs(r400[c]) / abs(r100[c]) < 0.3
        assert abs(r400[c]) < 1e-3 * abs(g400[c])
    # planted mistake: the image added instead of subtracted
    real = og.extracted_part

    def wrong_image(kx, ky, eps_eff, h, k0_):
        kx = np.asarray(kx, dtype=np.complex128)
        ky = np.asarray(ky, dtype=np.complex128)
        beta_sq = kx * kx + ky * ky
        kz = og.kz_free(beta_sq, np.sqrt(eps_eff) * k0_)
        f = 1.0 + np.exp(-2j * kz * h)
        z_te = k0_ * og.Z0 * f / (2.0 * kz)
        z_tm = og.Z0 * kz * f / (2.0 * k0_ * eps_eff)
        d = (z_tm - z_te) / beta_sq
        return -z_te - d * kx * kx, -d * kx * ky, -z_te - d * ky * ky

    og.extracted_part = wrong_image
    try:
        part = og.layered_remainder()(1.8, 2.4, 1.0, 0.05, k0)
        full = og.dyadic_green(1.8, 2.4, 1.0, 0.05, k0)
        assert abs(part[0]) > 0.1 * abs(full[0])
    finally:
        og.extracted_part = real
