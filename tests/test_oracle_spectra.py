"""Pins for the oracle's basis-function and MBF spectra.

Each closed form is checked against brute-force Gauss-Legendre quadrature of
the spatial current (Eq. 5 convention, F(k) = int f(r) exp(-i k.r) dr), at
real and complex wavenumbers (the analytic continuation of Eq. 18), including
the removable singularity of the strip transform.  The rotation rule is
checked against an explicitly rotated mesh.
"""
import math

import numpy as np
import pytest

from oracle import spectra

K0 = 2 * math.pi


def _gl(a, b, n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def brute_rooftop(kx, ky, cx, cy, direction, a, w):
    # along the current: two pieces (kink at 0); across: one piece
    u1, wu1 = _gl(-a, 0.0, 40)
    u2, wu2 = _gl(0.0, a, 40)
    u = np.concatenate([u1, u2])
    wu = np.concatenate([wu1, wu2])
    v, wv = _gl(-w / 2, w / 2, 40)
    prof = (1 - np.abs(u) / a)[:, None] / w * np.ones_like(v)[None, :]
    uu, vv = np.meshgrid(u, v, indexing="ij")
    if direction == 0:
        x, y = cx + uu, cy + vv
    else:
        x, y = cx + vv, cy + uu
    ph = np.exp(-1j * (kx * x + ky * y))
    return np.sum(prof * ph * wu[:, None] * wv[None, :])


def brute_strip(kx, ky, length, width):
    x, wx = _gl(-length / 2, length / 2, 80)
    y, wy = _gl(-width / 2, width / 2, 20)
    fx = np.sum(np.cos(np.pi * x / length) * np.exp(-1j * kx * x) * wx)
    fy = np.sum(np.exp(-1j * ky * y) * wy) / width
    return fx * fy


KPTS = [(0.0, 0.0), (3.1, -2.2), (12.0, 7.5), (40.0 + 0.3j, -25.0 + 0.1j), (0.2 + 0.05j, 9.0 - 0.02j)]


@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("k", KPTS)
def test_rooftop_closed_form(direction, k):
    kx, ky = k
    got = spectra.rooftop_ft(kx, ky, 0.12, -0.07, direction, 0.05, 0.03)
    ref = brute_rooftop(kx, ky, 0.12, -0.07, direction, 0.05, 0.03)
    assert abs(got - ref) < 1e-12 * max(1.0, abs(ref)) * 0.05


@pytest.mark.parametrize("k", KPTS + [(math.pi / 0.45, 1.0), (-math.pi / 0.45 + 1e-9, 0.0),
                                      (math.pi / 0.45 + 0.01j, 2.0)])
def test_strip_closed_form(k):
    kx, ky = k
    got = spectra.strip_ft(kx, ky, 0.45, 0.02)
    ref = brute_strip(kx, ky, 0.45, 0.02)
    assert abs(got - ref) < 1e-12 * max(abs(ref), 0.1)


def test_strip_removable_singularity_value():
    # F(kx = pi/L, ky = 0) = L/2 (limit of 2 pi L cos(u)/(pi^2 - 4u^2), u -> pi/2)
    assert abs(spectra.strip_ft(math.pi / 0.45, 0.0, 0.45, 0.02) - 0.45 / 2) < 1e-14


def _small_mesh(seed=7, m=2):
    rng = np.random.default_rng(seed)
    cx = np.array([-0.1, 0.0, 0.1, -0.05, 0.05, 0.07])
    cy = np.array([0.0, 0.05, -0.05, 0.1, -0.1, 0.02])
    d = np.array([0, 0, 0, 1, 1, 1])
    q = rng.standard_normal((6, m)) + 1j * rng.standard_normal((6, m))
    return spectra.BasisSet("rooftop", q, cx=cx, cy=cy, direction=d,
                            half_len=np.full(6, 0.05), width=np.full(6, 0.04))


def test_mbf_spectra_sum_of_conjugated_coefficients():
    # Eq. 11: M = sum_j conj(q_j) F_j, direction-resolved
    bs = _small_mesh()
    kx = np.array([1.0, 14.0 + 0.2j])
    ky = np.array([-3.0, 5.0 + 0.1j])
    mx, my = spectra.mbf_spectra(bs, kx, ky)
    for a in range(bs.n_mbf):
        ex = sum(np.conj(bs.q[i, a]) * brute_rooftop(kx[0], ky[0], bs.geom["cx"][i], bs.geom["cy"][i],
                                                      0, 0.05, 0.04)
                 for i in range(3))
        assert abs(mx[a, 0] - ex) < 1e-12 * abs(ex)
    # conjugate side: Mbar(k) = sum q F(-k)
    bx, by = spectra.mbf_spectra(bs, kx, ky, conjugate_side=True)
    for a in range(bs.n_mbf):
        ey = sum(bs.q[i, a] * brute_rooftop(-kx[1], -ky[1], bs.geom["cx"][i], bs.geom["cy"][i],
                                            1, 0.05, 0.04)
                 for i in range(3, 6))
        assert abs(by[a, 1] - ey) < 1e-12 * abs(ey)
    # on real k, Mbar = conj(M) for real currents
    mx2, my2 = spectra.mbf_spectra(bs, kx[:1], ky[:1])
    bx2, by2 = spectra.mbf_spectra(bs, kx[:1], ky[:1], conjugate_side=True)
    assert np.allclose(bx2, np.conj(mx2), rtol=1e-13) and np.allclose(by2, np.conj(my2), rtol=1e-13)


def test_rotation_matches_explicitly_rotated_mesh():
    bs = _small_mesh()
    g = bs.geom
    # rotate by +90 deg: centre (x, y) -> (-y, x); x-current -> +y; y-current -> -x
    d = g["direction"]
    sign = np.where(d == 1, -1.0, 1.0)
    rot = spectra.BasisSet("rooftop", bs.q * sign[:, None], cx=-g["cy"], cy=g["cx"],
                           direction=1 - d, half_len=g["half_len"], width=g["width"])
    kx = np.array([2.0, 11.0 + 0.1j, -7.0])
    ky = np.array([5.0, -3.0 + 0.05j, 0.5])
    for conj_side in (False, True):
        a = spectra.mbf_spectra(bs, kx, ky, theta=math.pi / 2, conjugate_side=conj_side)
        b = spectra.mbf_spectra(rot, kx, ky, conjugate_side=conj_side)
        assert np.allclose(a[0], b[0], rtol=1e-12, atol=1e-13)
        assert np.allclose(a[1], b[1], rtol=1e-12, atol=1e-13)
