"""The oracle's pins catch plausible mistakes.

Each test plants one mistake in the oracle (on the CPU, through monkeypatch)
-- a dropped contour Jacobian, a flipped off-diagonal Green's term, a
conjugate on the wrong side, a (+i)^q instead of (-i)^q, a transposed
rotation, a wrong free-space branch, a reversed separation vector, a diagonal
Green's term copied from the other, a dropped radial measure, the opposite
sign of the harmonic transform -- and checks that the quantity the
corresponding pin asserts moves far outside that pin's tolerance.
"""
import math

import numpy as np

from oracle import contour, green, reaction, spectra

K0 = 2 * math.pi


def gaussian_hankel_error():
    """Richardson-extrapolated error of the Gaussian Hankel pair (pin: < 1e-9)."""
    q, s = 1, 0.35
    rho = np.array([0.4, 1.3])
    exact = ((-1j) ** q / (2 * np.pi)) * rho ** q / (2 * s * s) ** (q + 1) * np.exp(-rho ** 2 / (4 * s * s))
    zs = []
    for n in (1000, 2000):
        c = contour.contour_nodes(n, 30.0, 8.1, 0.6)
        hq = (c["beta_c"] * np.exp(-s * s * c["beta_c"] ** 2))[None, :]
        zs.append(reaction.table_bessel(hq, [q], c["beta_c"], c["weight"], rho)[0])
    rich = (4 * zs[1] - zs[0]) / 3
    return np.abs(rich - exact).max() / np.abs(exact).max()


def rotational_covariance_error():
    """max |G(Rk) - R G(k) R^T| / |G| (pin: < 1e-12)."""
    k = np.array([1.3 * K0 + 0.02j, 0.7 * K0 + 0.01j])
    th = 0.7
    r = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    g = np.array(green.dyadic_green(k[0], k[1], 4.4, 0.03, K0))
    g = np.array([[g[0], g[1]], [g[1], g[2]]])
    rk = r @ k
    g2 = np.array(green.dyadic_green(rk[0], rk[1], 4.4, 0.03, K0))
    g2 = np.array([[g2[0], g2[1]], [g2[1], g2[2]]])
    return np.abs(g2 - r @ g @ r.T).max() / np.abs(g).max()


def _patch(seed=11):
    rng = np.random.default_rng(seed)
    ax = np.array([-0.1, 0.0, 0.1])
    gx, gy = np.meshgrid(ax, ax)
    cx = np.concatenate([gx.ravel(), gx.ravel()])
    cy = np.concatenate([gy.ravel(), gy.ravel()])
    d = np.concatenate([np.zeros(9, int), np.ones(9, int)])
    q = rng.standard_normal((18, 2)) + 1j * rng.standard_normal((18, 2))
    return spectra.BasisSet("rooftop", q, cx=cx, cy=cy, direction=d, half_len=np.full(18, 0.1),
                            width=np.full(18, 0.1))


def reciprocity_error():
    """|Z_ab,q[Q] - (-1)^q Z_ba,q[conj Q]| / max|Z| (pin: < 1e-11)."""
    kd = K0 * math.sqrt(4.4)
    c = contour.contour_nodes(300, 5 * kd, 1.3 * kd, 6 * 5 * kd / 300)
    bs = _patch()
    bsc = spectra.BasisSet("rooftop", np.conj(bs.q), **bs.geom)
    qs = np.arange(-3, 4)
    rho = np.array([0.3, 1.2])
    z = reaction.table_bessel(reaction.harmonics(bs, c["beta_c"], qs, 64, 4.4, 0.03, K0), qs,
                              c["beta_c"], c["weight"], rho)
    zc = reaction.table_bessel(reaction.harmonics(bsc, c["beta_c"], qs, 64, 4.4, 0.03, K0), qs,
                               c["beta_c"], c["weight"], rho)
    sign = ((-1.0) ** np.abs(qs))[:, None]
    return np.abs(z - np.swapaxes(zc, 0, 1) * sign).max() / np.abs(z).max()


def gaussian_2d_error():
    """Z'(rho, phi) of two Gaussian currents vs the 2-D Fourier pair (pin: < 1e-10)."""
    s = 0.12
    c0, c1 = np.array([0.05, -0.03]), np.array([-0.04, 0.02])
    bs = spectra.BasisSet("gaussian", np.eye(2), cx=np.array([c0[0], c1[0]]),
                          cy=np.array([c0[1], c1[1]]), direction=np.array([0, 0]), s=s)
    qs = np.arange(-14, 15)
    c = contour.contour_nodes(3000, 45.0, 9.9, 0.5)
    hq = reaction.harmonics(bs, c["beta_c"], qs, 64, 0, 0, K0, green_fn=green.identity_green)
    zq = reaction.table_bessel(hq, qs, c["beta_c"], c["weight"], np.array([0.3]))[..., 0]
    phi = 1.0
    z = reaction.reaction_from_table(zq, qs, phi)
    d = 0.3 * np.array([math.cos(phi), math.sin(phi)]) + c0 - c1
    exact = np.exp(-d @ d / (8 * s * s)) / (8 * np.pi * s * s)
    return abs(z[0, 1] - exact) / exact


def rotation_error():
    """spectra at theta = 90 deg vs an explicitly rotated mesh (pin: < 1e-12)."""
    bs = _patch()
    g = bs.geom
    d = g["direction"]
    sign = np.where(d == 1, -1.0, 1.0)
    rot = spectra.BasisSet("rooftop", bs.q * sign[:, None], cx=-g["cy"], cy=g["cx"], direction=1 - d,
                           half_len=g["half_len"], width=g["width"])
    kx, ky = np.array([2.0, 11.0 + 0.1j]), np.array([5.0, -3.0 + 0.05j])
    a = spectra.mbf_spectra(bs, kx, ky, theta=math.pi / 2)
    b = spectra.mbf_spectra(rot, kx, ky)
    return max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()) / np.abs(b[0]).max()


def test_unmutated_oracle_meets_every_pin():
    assert gaussian_hankel_error() < 1e-9
    assert rotational_covariance_error() < 1e-12
    assert reciprocity_error() < 1e-11
    assert gaussian_2d_error() < 1e-5   # single resolution here (no Richardson): O(h^2)
    assert rotation_error() < 1e-12


def test_dropped_contour_jacobian_is_caught(monkeypatch):
    orig = contour.contour_nodes

    def no_jacobian(n, beta_max, beta_p, height):
        d = orig(n, beta_max, beta_p, height)
        d["weight"] = np.full(n, d["h"], dtype=np.complex128)
        return d

    monkeypatch.setattr(contour, "contour_nodes", no_jacobian)
    assert gaussian_hankel_error() > 1e-3


def test_flipped_off_diagonal_green_is_caught(monkeypatch):
    orig = green.dyadic_green
    monkeypatch.setattr(green, "dyadic_green",
                        lambda kx, ky, e, h, k0: (lambda g: (g[0], -g[1], g[2]))(orig(kx, ky, e, h, k0)))
    assert rotational_covariance_error() > 1e-3


def test_conjugate_on_both_sides_is_caught(monkeypatch):
    orig = spectra.mbf_spectra

    def both_conj(basis, kx, ky, theta=0.0, conjugate_side=False):
        if conjugate_side:
            b2 = spectra.BasisSet(basis.kind, np.conj(basis.q), **basis.geom)
            return orig(b2, kx, ky, theta=theta, conjugate_side=True)
        return orig(basis, kx, ky, theta=theta, conjugate_side=False)

    monkeypatch.setattr(spectra, "mbf_spectra", both_conj)
    assert reciprocity_error() > 1e-3


def test_wrong_harmonic_phase_is_caught(monkeypatch):
    orig = reaction.table_bessel

    def plus_i(hq, qs, beta_c, weight, rho):
        z = orig(hq, qs, beta_c, weight, rho)
        fix = np.array([(1j) ** int(q) / (-1j) ** int(q) for q in qs])
        return z * fix.reshape((1,) * (z.ndim - 2) + (-1, 1))

    monkeypatch.setattr(reaction, "table_bessel", plus_i)
    assert gaussian_2d_error() > 1e-2


def test_transposed_rotation_is_caught(monkeypatch):
    orig = spectra._rotate_k
    monkeypatch.setattr(spectra, "_rotate_k", lambda kx, ky, th: orig(kx, ky, -th))
    assert rotation_error() > 1e-3


def test_wrong_free_space_branch_is_caught(monkeypatch):
    # k2 with Im k2 >= 0 (growing field) instead of the radiation condition
    monkeypatch.setattr(green, "_branch_sqrt_free", lambda w: 1j * np.sqrt(np.asarray(w, dtype=np.complex128)))
    bc = np.array([0.5, 1.5]) * K0 + 0.05j
    assert np.any(green.kz_free(bc ** 2, K0).imag > 0)   # the radiation-condition pin fails


def test_reversed_separation_is_caught(monkeypatch):
    # Delta = r_basis - r_test instead of r_test - r_basis: phi -> phi + pi
    orig = reaction.reaction_from_table
    monkeypatch.setattr(reaction, "reaction_from_table", lambda zq, qs, phi: orig(zq, qs, phi + math.pi))
    assert gaussian_2d_error() > 1e-2


def test_copied_diagonal_green_term_is_caught(monkeypatch):
    # Gyy written as a copy of Gxx (kx where ky belongs)
    orig = green.dyadic_green
    monkeypatch.setattr(green, "dyadic_green",
                        lambda kx, ky, e, h, k0: (lambda g: (g[0], g[1], g[0]))(orig(kx, ky, e, h, k0)))
    assert rotational_covariance_error() > 1e-3


def test_dropped_radial_measure_is_caught(monkeypatch):
    # the beta of beta d beta left out of the radial quadrature
    orig = reaction.table_bessel
    monkeypatch.setattr(reaction, "table_bessel",
                        lambda hq, qs, beta_c, weight, rho: orig(np.asarray(hq) / beta_c, qs, beta_c, weight, rho))
    assert gaussian_hankel_error() > 1e-3


def test_harmonic_sign_convention_is_caught(monkeypatch):
    # H_q taken with exp(+i q alpha) instead of exp(-i q alpha): q -> -q (the q list is symmetric)
    orig = reaction.harmonics
    monkeypatch.setattr(reaction, "harmonics", lambda *a, **k: orig(*a, **k)[..., ::-1, :])
    assert gaussian_2d_error() > 1e-2


def gaussian_array_error():
    """Reduced matrix of a 3-element array of x- and y-directed Gaussian currents
    (rotations 0/90) under a unit dyadic vs its closed form (the pin of
    test_oracle_fill.py, one resolution)."""
    from oracle import fill
    s = 0.1
    cs = np.array([[0.04, -0.02], [-0.03, 0.05]])
    dirs = np.array([[1.0, 0.0], [0.0, 1.0]])
    bs = spectra.BasisSet("gaussian", np.eye(2), cx=cs[:, 0], cy=cs[:, 1], direction=np.array([0, 1]), s=s)
    pos = np.array([[0.0, 0.0], [0.25, 0.1], [-0.12, 0.3]])
    rot = np.array([0, 1, 0])
    qs = np.arange(-16, 17)
    c = contour.contour_nodes(2000, 60.0, 12.0, 0.4)
    hq = {cls: reaction.harmonics(bs, c["beta_c"], qs, 96, 0, 0, K0, *reaction.rotation_angles(cls),
                                  green_fn=green.identity_green) for cls in range(4)}
    z = fill.full_matrix(hq, qs, c["beta_c"], c["weight"], pos, rot)

    def rmat(t):
        return np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])
    exact = np.empty_like(z)
    for m in range(3):
        for n in range(3):
            tm, tn = rot[m] * math.pi / 2, rot[n] * math.pi / 2
            for a in range(2):
                for b in range(2):
                    d = pos[m] - pos[n] + rmat(tm) @ cs[a] - rmat(tn) @ cs[b]
                    align = (rmat(tm) @ dirs[a]) @ (rmat(tn) @ dirs[b])
                    exact[2 * m + a, 2 * n + b] = align * math.exp(-d @ d / (8 * s * s)) / (8 * math.pi * s * s)
    return np.abs(z - exact).max() * 8 * math.pi * s * s


def rooftop_error():
    """Closed-form rooftop transform vs Gauss-Legendre quadrature of the current (pin: 1e-12)."""
    from tests.test_oracle_spectra import brute_rooftop
    worst = 0.0
    for kx, ky in ((3.1, -2.2), (12.0, 7.5), (40.0 + 0.3j, -25.0 + 0.1j)):
        got = spectra.rooftop_ft(kx, ky, 0.12, -0.07, 0, 0.05, 0.03)
        ref = brute_rooftop(kx, ky, 0.12, -0.07, 0, 0.05, 0.03)
        worst = max(worst, abs(got - ref) / abs(ref))
    return worst


def test_unmutated_fill_and_rooftop_meet_their_pins():
    assert gaussian_array_error() < 1e-4      # one resolution: O(h^2) quadrature error
    assert rooftop_error() < 1e-10


def test_swapped_rotation_class_is_caught(monkeypatch):
    from oracle import fill
    monkeypatch.setattr(fill, "class_index", lambda rot, m, n: 2 * int(rot[n]) + int(rot[m]))
    assert gaussian_array_error() > 1e-2


def test_swapped_pair_geometry_is_caught(monkeypatch):
    from oracle import fill
    orig = fill.pair_geometry
    monkeypatch.setattr(fill, "pair_geometry", lambda pos, m, n: orig(pos, n, m))
    assert gaussian_array_error() > 1e-2


def test_rooftop_with_a_single_sinc_is_caught(monkeypatch):
    def one_sinc(kx, ky, cx, cy, direction, half_len, width):
        kx = np.asarray(kx, dtype=np.complex128)
        ky = np.asarray(ky, dtype=np.complex128)
        ku, kv = (kx, ky) if direction == 0 else (ky, kx)
        shape = half_len * spectra.sinc(ku * half_len / 2.0) * spectra.sinc(kv * width / 2.0)
        return np.exp(-1j * (kx * cx + ky * cy)) * shape
    monkeypatch.setattr(spectra, "rooftop_ft", one_sinc)
    assert rooftop_error() > 1e-3


def tl_model_error():
    """max |G - G_TL| / |G_TL| against the transmission-line derivation (pin: 1e-11)."""
    from tests.test_oracle_green import tl_dyadic
    eps_r, h = 4.4, 0.03
    betas = np.array([0.5, 1.3, 2.4, 9.0]) * K0 + 0.02j
    kx, ky = betas * math.cos(0.7), betas * math.sin(0.7)
    got = green.dyadic_green(kx, ky, eps_r, h, K0)
    ref = tl_dyadic(kx, ky, eps_r, h, K0, green.Z0)
    scale = np.maximum(np.abs(ref[0]), np.abs(ref[2]))
    return max(np.max(np.abs(g - r) / scale) for g, r in zip(got, ref))


def test_consistent_numerator_sign_slip_is_caught(monkeypatch):
    # the j k1 sin(k1 h) terms of every numerator with the opposite sign: the dyadic stays
    # covariant, its leading thin-slab terms and its poles are unchanged -- only the
    # transmission-line pin sees it
    def slipped(kx, ky, eps_r, h, k0):
        kx = np.asarray(kx, dtype=np.complex128)
        ky = np.asarray(ky, dtype=np.complex128)
        b2 = kx * kx + ky * ky
        k1, k2 = green.kz_slab(b2, eps_r, k0), green.kz_free(b2, k0)
        c, s = np.cos(k1 * h), np.sin(k1 * h)
        te, tm = green.te_tm(b2, eps_r, h, k0)
        common = s / (te * tm)
        z = -1j * green.Z0 / k0
        gxx = z * ((eps_r * k0 ** 2 - kx * kx) * k2 * c - 1j * (k0 ** 2 - kx * kx) * k1 * s) * common
        gyy = z * ((eps_r * k0 ** 2 - ky * ky) * k2 * c - 1j * (k0 ** 2 - ky * ky) * k1 * s) * common
        gxy = -z * kx * ky * (k2 * c - 1j * k1 * s) * common
        return gxx, gxy, gyy
    assert tl_model_error() < 1e-11
    monkeypatch.setattr(green, "dyadic_green", slipped)
    assert rotational_covariance_error() < 1e-12      # the covariance pin does not see it
    assert tl_model_error() > 1e-3
