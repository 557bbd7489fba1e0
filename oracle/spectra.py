"""Fourier transforms of elementary basis functions and of MBFs (Eq. 11).

Convention (Eq. 5): F(k) = integral of f(r) exp(-i k.r) dr, evaluated at
complex kx, ky by analytic continuation (Eq. 18).  Each basis function is a
surface current with a fixed direction (x or y) and the closed-form transform
the paper says is available for rooftops (Section III-A):

* rooftop, direction d, centre c, half-length a, width w:
    current (1 - |u|/a)/w on |u| <= a (along d), |v| <= w/2 (across d)
    F(k) = exp(-i k.c) * a sinc^2(k_u a / 2) * sinc(k_v w / 2)
* strip dipole (centre 0, along x, length L, width W):
    current cos(pi x / L)/W on |x| <= L/2, |y| <= W/2
    F(k) = 2 pi L cos(kx L/2) / (pi^2 - kx^2 L^2) * sinc(ky W / 2)
* gaussian (test basis, centre c, width s, along d):
    F(k) = exp(-s^2 (kx^2 + ky^2)) exp(-i k.c)

with sinc(z) = sin(z)/z.  MBF spectra follow Eq. 11 with conjugated
coefficients, M_a(k) = sum_i conj(Q_ia) F_i(k) d_i, and the conjugated basis
spectrum of Eq. 10 continues analytically as Mbar_b(k) = sum_i Q_ib F_i(-k) d_i
(equal to conj(M_b(k)) on real k for real currents).

A rotated element (angle theta, rotation matrix R) has M^theta(k) = R M(R^T k).

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np


def sinc(z):
    """sin(z)/z for complex z, with the Taylor series near 0."""
    z = np.asarray(z, dtype=np.complex128)
    small = np.abs(z) < 1e-3
    safe = np.where(small, 1.0, z)
    z2 = z * z
    series = 1.0 - z2 / 6.0 + z2 * z2 / 120.0 - z2 * z2 * z2 / 5040.0
    return np.where(small, series, np.sin(safe) / safe)


def rooftop_ft(kx, ky, cx, cy, direction, half_len, width):
    """Transform of one rooftop (direction 0 = x, 1 = y)."""
    kx = np.asarray(kx, dtype=np.complex128)
    ky = np.asarray(ky, dtype=np.complex128)
    ku, kv = (kx, ky) if direction == 0 else (ky, kx)
    shape = half_len * sinc(ku * half_len / 2.0) ** 2 * sinc(kv * width / 2.0)
    return np.exp(-1j * (kx * cx + ky * cy)) * shape


def strip_ft(kx, ky, length, width):
    """Transform of the x-directed cosine strip dipole centred at the origin.

    The removable singularities at kx L = +-pi are handled by writing
    cos(u) / (pi^2/4 - u^2) = sinc(pi/2 - u) / (pi/2 + u), u = kx L / 2,
    mirrored for Re u < 0 (the factor is even in u).
    """
    kx = np.asarray(kx, dtype=np.complex128)
    ky = np.asarray(ky, dtype=np.complex128)
    u = kx * length / 2.0
    u = np.where(u.real < 0.0, -u, u)
    along = (np.pi * length / 2.0) * sinc(np.pi / 2.0 - u) / (np.pi / 2.0 + u)
    return along * sinc(ky * width / 2.0)


def gaussian_ft(kx, ky, cx, cy, s):
    """Transform of a Gaussian test current (entire in kx, ky)."""
    kx = np.asarray(kx, dtype=np.complex128)
    ky = np.asarray(ky, dtype=np.complex128)
    return np.exp(-s * s * (kx * kx + ky * ky)) * np.exp(-1j * (kx * cx + ky * cy))


class BasisSet:
    """Elementary basis functions of one element plus its MBF coefficient matrix Q.

    kind: "rooftop" (arrays cx, cy, direction, half_len, width of length B),
          "strip"   (scalars length, width; B = 1, x-directed),
          "gaussian"(arrays cx, cy, direction, s).
    q:    complex (B, M) matrix whose columns are the MBFs (Eq. 3).
    """

    def __init__(self, kind, q, **geom):
        self.kind = kind
        self.q = np.asarray(q, dtype=np.complex128)
        self.geom = {k: (np.asarray(v) if np.ndim(v) else v) for k, v in geom.items()}
        if self.q.ndim != 2:
            raise ValueError("q must be (B, M)")

    @property
    def n_basis(self):
        return self.q.shape[0]

    @property
    def n_mbf(self):
        return self.q.shape[1]

    def all_ft(self, kx, ky):
        """Transforms of every basis function: (F, d) with F of shape
        (B,) + broadcast(kx, ky).shape and d the direction of each (0 = x, 1 = y)."""
        g = self.geom
        kx = np.asarray(kx, dtype=np.complex128)[None]
        ky = np.asarray(ky, dtype=np.complex128)[None]
        if self.kind == "strip":
            return strip_ft(kx, ky, g["length"], g["width"]), np.zeros(1, dtype=int)
        ext = (slice(None),) + (None,) * (kx.ndim - 1)
        cx, cy = g["cx"][ext], g["cy"][ext]
        d = np.asarray(g["direction"], dtype=int)
        if self.kind == "rooftop":
            a, w = g["half_len"][ext], g["width"][ext]
            is_x = (d == 0)[ext]
            ku = np.where(is_x, kx, ky)
            kv = np.where(is_x, ky, kx)
            shape = a * sinc(ku * a / 2.0) ** 2 * sinc(kv * w / 2.0)
            return np.exp(-1j * (kx * cx + ky * cy)) * shape, d
        if self.kind == "gaussian":
            return gaussian_ft(kx, ky, cx, cy, g["s"]), d
        raise ValueError(self.kind)


def _rotate_k(kx, ky, theta):
    """R^T k for the rotation R by theta (counter-clockwise)."""
    c, s = np.cos(theta), np.sin(theta)
    return c * kx + s * ky, -s * kx + c * ky


def _rotate_vec(vx, vy, theta):
    c, s = np.cos(theta), np.sin(theta)
    return c * vx - s * vy, s * vx + c * vy


def mbf_spectra(basis, kx, ky, theta=0.0, conjugate_side=False):
    """Vector MBF spectra at (kx, ky).

    conjugate_side=False: M_a(k) = sum_i conj(Q_ia) F_i(k) d_i      (Eq. 11)
    conjugate_side=True : Mbar_b(k) = sum_i Q_ib F_i(-k) d_i       (Eq. 10, M_b^*)
    theta: element rotation; returns R M(R^T k).
    Returns (Mx, My), each of shape (M,) + broadcast(kx, ky).shape.
    """
    kx = np.asarray(kx, dtype=np.complex128)
    ky = np.asarray(ky, dtype=np.complex128)
    kxr, kyr = _rotate_k(kx, ky, theta)
    if conjugate_side:
        kxr, kyr = -kxr, -kyr
        coef = basis.q
    else:
        coef = np.conj(basis.q)
    f, d = basis.all_ft(kxr, kyr)                      # (B, ...)
    shape = f.shape[1:]
    flat = f.reshape(f.shape[0], -1)
    cx = np.where((d == 0)[:, None], coef, 0.0)        # (B, M) weights of x-directed bases
    cy = np.where((d == 1)[:, None], coef, 0.0)
    mx = (cx.T @ flat).reshape((basis.n_mbf,) + shape)  # sum over i of coef_ia F_i
    my = (cy.T @ flat).reshape((basis.n_mbf,) + shape)
    if theta != 0.0:
        mx, my = _rotate_vec(mx, my, theta)
    return mx, my
