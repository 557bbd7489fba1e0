"""Spectral dyadic Green's function of a grounded dielectric slab (FP64).

The paper uses the layered-medium dyadic Green's function G~ in Eq. 6 and
Eq. 10 (Section III-A) and cites its standard form without printing it.  The
form used here is the classical one for the tangential electric field at the
top of a grounded slab (relative permittivity eps_r, thickness h, free space
above) due to a horizontal electric surface current at the same interface,
with an exp(+j omega t) time convention (the paper's ``i`` is read as ``j``):

    k2 = sqrt(k0^2 - beta^2),  Im k2 <= 0   (free space, outgoing/decaying)
    k1 = sqrt(eps_r k0^2 - beta^2)          (slab; G is even in k1, any branch)
    Te = k1 cos(k1 h) + j k2 sin(k1 h)      (TE surface-wave denominator)
    Tm = eps_r k2 cos(k1 h) + j k1 sin(k1 h)(TM surface-wave denominator)
    Gxx = -j Z0/k0 [(eps_r k0^2 - kx^2) k2 cos + j (k0^2 - kx^2) k1 sin] sin / (Te Tm)
    Gxy = Gyx = +j Z0/k0 kx ky [k2 cos + j k1 sin] sin / (Te Tm)
    Gyy = Gxx with kx <-> ky

with cos = cos(k1 h), sin = sin(k1 h), beta^2 = kx^2 + ky^2 (no conjugation,
so the same expressions continue analytically to complex kx, ky as Eq. 18
requires).  The surface-wave poles are the zeros of Te and Tm; the paper's
contour (Eq. 8) passes above them.  ``dyadic_green`` extracts nothing;
``layered_remainder`` subtracts an effective homogeneous medium and its image
through the ground plane (``extracted_part``), the split of Section II.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import math

import numpy as np

# Free-space wave impedance (ohm), sqrt(mu0 / eps0).
Z0 = 376.730313668


def _branch_sqrt_free(w):
    """-j * sqrt(w) with the principal root; for w exactly on the negative real
    axis the root is taken from the upper side (k2 real positive, outgoing)."""
    w = np.asarray(w, dtype=np.complex128)
    on_axis = w.imag == 0.0
    w = np.where(on_axis, w.real + 0.0j, w)
    return -1j * np.sqrt(w)


def kz_free(beta_sq, k0):
    """Free-space vertical wavenumber k2 = sqrt(k0^2 - beta^2) with Im k2 <= 0."""
    return _branch_sqrt_free(np.asarray(beta_sq, dtype=np.complex128) - k0 ** 2)


def kz_slab(beta_sq, eps_r, k0):
    """Slab vertical wavenumber k1 = sqrt(eps_r k0^2 - beta^2) (principal root)."""
    return np.sqrt(eps_r * k0 ** 2 - np.asarray(beta_sq, dtype=np.complex128))


def te_tm(beta_sq, eps_r, h, k0):
    """TE and TM denominators (Te, Tm) at radial wavenumber squared beta_sq."""
    k1 = kz_slab(beta_sq, eps_r, k0)
    k2 = kz_free(beta_sq, k0)
    c = np.cos(k1 * h)
    s = np.sin(k1 * h)
    te = k1 * c + 1j * k2 * s
    tm = eps_r * k2 * c + 1j * k1 * s
    return te, tm


def dyadic_green(kx, ky, eps_r, h, k0):
    """Return (Gxx, Gxy, Gyy) of the grounded slab at (possibly complex) kx, ky."""
    kx = np.asarray(kx, dtype=np.complex128)
    ky = np.asarray(ky, dtype=np.complex128)
    beta_sq = kx * kx + ky * ky
    k1 = kz_slab(beta_sq, eps_r, k0)
    k2 = kz_free(beta_sq, k0)
    c = np.cos(k1 * h)
    s = np.sin(k1 * h)
    te = k1 * c + 1j * k2 * s
    tm = eps_r * k2 * c + 1j * k1 * s
    common = s / (te * tm)
    gxx = (-1j * Z0 / k0) * ((eps_r * k0 ** 2 - kx * kx) * k2 * c
                             + 1j * (k0 ** 2 - kx * kx) * k1 * s) * common
    gyy = (-1j * Z0 / k0) * ((eps_r * k0 ** 2 - ky * ky) * k2 * c
                             + 1j * (k0 ** 2 - ky * ky) * k1 * s) * common
    gxy = (1j * Z0 / k0) * kx * ky * (k2 * c + 1j * k1 * s) * common
    return gxx, gxy, gyy


def identity_green(kx, ky, *unused):
    """Unit dyadic (test mode: isolates the transform from the substrate)."""
    one = np.ones(np.broadcast(np.asarray(kx), np.asarray(ky)).shape, dtype=np.complex128)
    return one, 0.0 * one, one


def extracted_part(kx, ky, eps_eff, h, k0):
    """The effective homogeneous medium and its image through the ground plane (the part
    of the slab Green's function that Sections II and III-A assign to Z^h).  Reading: a
    current sheet in a homogeneous medium of permittivity eps_eff (mu_0), ground plane h
    below: the medium's matched line in parallel with its line shorted at distance h,
      Z = Z_c (1 - exp(-2 j kz h)) / 2,  Z_c^TE = k0 Z0 / kz,  Z_c^TM = Z0 kz / (k0 eps_eff),
    kz = -j sqrt(beta^2 - eps_eff k0^2), in the dyadic -Z_TE I - (Z_TM - Z_TE) k k^T / beta^2.
    Returns (Gxx, Gxy, Gyy)."""
    kx = np.asarray(kx, dtype=np.complex128)
    ky = np.asarray(ky, dtype=np.complex128)
    beta_sq = kx * kx + ky * ky
    kz = kz_free(beta_sq, math.sqrt(eps_eff) * k0)
    f = 1.0 - np.exp(-2j * kz * h)
    z_te = k0 * Z0 * f / (2.0 * kz)
    # (Z_TM - Z_TE) / beta^2 with kz^2 - eps_eff k0^2 = -beta^2: finite at beta = 0
    d = -Z0 * f / (2.0 * k0 * eps_eff * kz)
    return -z_te - d * kx * kx, -d * kx * ky, -z_te - d * ky * ky


def layered_remainder(eps_eff=None):
    """Green's function of Z^l (Section II): the slab's dyadic minus ``extracted_part``,
    with eps_eff = (eps_r + 1) / 2 unless given.  Same call signature as dyadic_green."""
    def green(kx, ky, eps_r, h, k0):
        e = 0.5 * (eps_r + 1.0) if eps_eff is None else eps_eff
        gxx, gxy, gyy = dyadic_green(kx, ky, eps_r, h, k0)
        exx, exy, eyy = extracted_part(kx, ky, e, h, k0)
        return gxx - exx, gxy - exy, gyy - eyy
    return green
