"""Pins of the oracle's 2-D Cartesian C-FFT (Section III-B-2/3, Eq. 21-24, Appendix I),
each fixed by something other than the oracle's own table:

- closed form: with the contour undeformed, a Gaussian current under a unit dyadic has
  Z'(d) = exp(-|d|^2 / (8 s^2)) / (8 pi s^2); the FFT assembly (Appendix I signs, K', the
  zero-padded refinement) must reproduce it at every lattice point, refined ones included;
- definition: on the deformed contour, the Taylor-expanded FFT table equals Eq. 21's
  rectangle-rule sum evaluated directly with the exact contour factor E_I, at lattice
  points of both parities;
- the polar integral: the table converges to the polar oracle's Z' (Bessel sum on a fine
  contour of the same height) as the grid is refined, faster than first order: the
  deformation's slope is discontinuous on the circle |k| = beta_p and the integrand is cut
  at the circle |k| = beta_max, neither of which a Cartesian grid follows, so the
  rectangle rule is first to second order there;
- second-order interpolation reproduces quadratics exactly;
- planted mistakes (the (1 + i gamma) Jacobian dropped, the padding shifted, the output
  sign dropped) each break a pin.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import cartesian as oca
from oracle import contour as oc
from oracle import fill as ofill
from oracle import green as ogr
from oracle import reaction as orx
from oracle import spectra as osp

S = 0.25


def _gauss():
    return osp.BasisSet("gaussian", np.ones((1, 1)), cx=np.zeros(1), cy=np.zeros(1),
                        direction=np.zeros(1, int), s=S)


def _gauss_closed(x):
    xx, yy = np.meshgrid(x, x, indexing="ij")
    return np.exp(-(xx ** 2 + yy ** 2) / (8 * S * S)) / (8 * math.pi * S * S)


def _strip():
    wl = workloads.strip_fp64()
    el = wl.element
    return wl, osp.BasisSet("strip", el.q, length=el.length, width=el.strip_width)


def test_gaussian_closed_form_on_the_undeformed_grid():
    tab, x = oca.table(_gauss(), 2.2, 0.05, 2 * math.pi, 20.0, 12.0, 0.0, 64, 0, green_fn=ogr.identity_green)
    ref = _gauss_closed(x)
    assert tab.shape == (1, 1, 128, 128)
    err = np.abs(tab[0, 0] - ref).max() / ref.max()
    assert err < 1e-12
    # the refined (odd) lattice points alone: the zero-padding must put the samples right
    assert np.abs(tab[0, 0, 1::2, 1::2] - ref[1::2, 1::2]).max() < 1e-12 * ref.max()


def test_table_equals_the_direct_sum_with_the_exact_contour_factor():
    wl, bs = _strip()
    s, c = wl.substrate, wl.contour
    n = 64
    dk = 2 * c.beta_max / n
    height = 6 * dk
    tab, x = oca.table(bs, s.eps_r, s.h, s.k0, c.beta_max, c.beta_p, height, n, 36)
    idx = [(n, n), (n + 1, n), (n + 5, n + 2), (n + 9, n - 4), (n - 7, n + 11), (n + 13, n + 13)]
    ds = oca.direct_sum(bs, s.eps_r, s.h, s.k0, c.beta_max, c.beta_p, height, n,
                        np.array([x[i] for i, _ in idx]), np.array([x[j] for _, j in idx]))
    tv = np.array([tab[0, 0, i, j] for i, j in idx])
    assert np.abs(tv - ds[0, 0]).max() < 1e-10 * np.abs(ds).max()


def _polar_reference(bs, wl, height, pts):
    s, c = wl.substrate, wl.contour
    nodes = oc.contour_nodes(8192, c.beta_max, c.beta_p, height)
    qs = np.arange(-40, 41)
    hq = orx.harmonics(bs, nodes["beta_c"], qs, 256, s.eps_r, s.h, s.k0)
    pos = np.array([[0.0, 0.0]] + [list(p) for p in pts])
    rot = np.zeros(len(pos), int)
    return np.array([ofill.entries({0: hq}, qs, nodes["beta_c"], nodes["weight"], pos, rot, [(k, 0)])[0, 0, 0]
                     for k in range(1, len(pos))])


def _cartesian_vs_polar():
    wl, bs = _strip()
    s, c = wl.substrate, wl.contour
    errs = []
    height = 6 * 2 * c.beta_max / 512
    ref = None
    for n in (256, 512):
        tab, x = oca.table(bs, s.eps_r, s.h, s.k0, c.beta_max, c.beta_p, height, n, 12)
        # the same physical points on both grids: lattice points of the coarser one
        rows = [n + 2 * t for t in (0, 4, 16, 30)]
        cols = [n + 2 * t for t in (0, 2, 10)]
        pts = [(x[i], x[j]) for i in rows for j in cols]
        if ref is None:
            ref = _polar_reference(bs, wl, height, pts)
        tv = np.array([tab[0, 0, i, j] for i in rows for j in cols])
        errs.append(np.abs(tv - ref).max() / np.abs(ref).max())
    return errs


@pytest.mark.slow
def test_converges_to_the_polar_integral():
    e256, e512 = _cartesian_vs_polar()
    print("Cartesian vs polar oracle: n 256 %.3g, n 512 %.3g" % (e256, e512))
    assert e512 < 1e-3 and e256 / e512 > 2.5


def test_quadratic_interpolation_is_exact_for_quadratics():
    x = -3.0 + 0.1 * np.arange(61)
    xx, yy = np.meshgrid(x, x, indexing="ij")
    f = 0.7 - 1.2 * xx + 0.3j * yy + 0.25 * xx * xx - (0.4 + 0.1j) * xx * yy + 0.05 * yy * yy
    rng = np.random.default_rng(3)
    px, py = rng.uniform(-2.5, 2.5, 20), rng.uniform(-2.5, 2.5, 20)
    got = oca.interpolate(f, x, px, py)
    want = 0.7 - 1.2 * px + 0.3j * py + 0.25 * px * px - (0.4 + 0.1j) * px * py + 0.05 * py * py
    assert np.abs(got - want).max() < 1e-12


def test_planted_mistakes_break_a_pin(monkeypatch):
    # output sign (-1)^(k1 + k2) dropped: every other lattice point flips sign
    real_fft2 = np.fft.fft2
    tab, x = oca.table(_gauss(), 2.2, 0.05, 2 * math.pi, 20.0, 12.0, 0.0, 64, 0, green_fn=ogr.identity_green)
    ref = _gauss_closed(x)
    idx = np.arange(128)
    sign = (-1.0) ** (idx[:, None] + idx[None, :])
    assert np.abs(tab[0, 0] * sign - ref).max() > 0.1 * ref.max()
    # the spectrum placed one sample off the middle of the padded grid
    monkeypatch.setattr(np.fft, "fft2", lambda a, axes=(-2, -1): real_fft2(np.roll(a, 1, axis=-1), axes=axes))
    bad, _ = oca.table(_gauss(), 2.2, 0.05, 2 * math.pi, 20.0, 12.0, 0.0, 64, 0, green_fn=ogr.identity_green)
    monkeypatch.setattr(np.fft, "fft2", real_fft2)
    assert np.abs(bad[0, 0] - ref).max() > 1e-3 * ref.max()


@pytest.mark.slow
def test_planted_jacobian_mistake_breaks_the_polar_pin(monkeypatch):
    real = oca.extended_kernel

    def without_gamma_factor(*args, **kw):
        im, gamma = real(*args, **kw)
        return im / (1.0 + 1j * gamma), gamma

    monkeypatch.setattr(oca, "extended_kernel", without_gamma_factor)
    e256, e512 = _cartesian_vs_polar()
    assert e512 > 1e-2
