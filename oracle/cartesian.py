"""The paper's 2-D Cartesian C-FFT (Section III-B-2 and III-B-3, Eq. 12-24; Appendix I).

The polar spectral integral of Eq. 9 is brought back to real rectangular
coordinates: with the analytic extension k_xI / k_xR = k_yI / k_yR = beta_I / beta_R
= gamma (Eq. 20), the deformed contour of Eq. 8 becomes, on the real (kx, ky) plane,

  Z'_ab(dx, dy) = 1/(4 pi^2) int int I_M(kx, ky) exp(-i (kx dx + ky dy)) E_I dkx dky   (Eq. 21)
  E_I = exp(gamma (kx dx + ky dy))
  I_M = (1 + i d beta_I / d beta_R) (1 + i gamma) H_ab(kx (1 + i gamma), ky (1 + i gamma))

with beta_R = |k| and H_ab the MBF kernel of Eq. 10.  The Taylor series of E_I (Eq. 22)
separates the spatial variables from the spectral ones:

  E_I = sum_n gamma^n (kx dx + ky dy)^n / n!
      = sum_{a, b} dx^a dy^b / (a! b!) (gamma kx)^a (gamma ky)^b,

so each monomial (a, b) is a plain 2-D Fourier sum (Eq. 23, the rectangle rule), and the
table is the Taylor-weighted sum of one FFT2 per monomial (Eq. 24).  Appendix I's change
of variables: on N x N spectral samples kx = -k_m + n1 dk (n1 = 0..N-1, dk = 2 k_m / N)
and spatial samples dx = -x_m + k1 pi / k_m (x_m = N pi / (2 k_m)),

  exp(-i kx dx) = exp(-i pi N / 2) (-1)^(n1 + k1) exp(-2 pi i n1 k1 / N),

so the FFT input carries (-1)^(n1 + n2), the output (-1)^(k1 + k2) and
K' = dk^2 / (4 pi^2); the global phase exp(-i pi N) of the two dimensions is 1 for even N.

The tables are refined by Whittaker-Shannon interpolation with zero padding to twice the
FFT size (the end of Section III-B-3): the spectral samples sit in the middle of a
2N x 2N grid of the same step, whose FFT2 gives the table at dx = -x_m + k1 pi / (2 k_m),
k1 = 0..2N-1; the fill interpolates that table with second-order (three-point) Lagrange
stencils in dx and dy.

Reading used here: the integrand is restricted to the disc |k| <= beta_max = k_m, the
hard truncation of the polar integral at 5 k_d (Section III-A), so that both
tabulations evaluate the same truncated integral; the paper's square spectral window
would add its corners.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import math

import numpy as np

from . import contour as _contour
from . import reaction as _reaction


def spectral_grid(n, k_max):
    """kx (= ky) samples of Appendix I: -k_m + n1 dk, n1 = 0..n-1, dk = 2 k_m / n."""
    dk = 2.0 * k_max / n
    return -k_max + dk * np.arange(n, dtype=np.float64), dk


def spatial_grid(n, k_max, refine=2):
    """dx (= dy) samples of the refined table: -x_m + k1 pi / (refine k_m), k1 < refine n."""
    x_m = n * math.pi / (2.0 * k_max)
    step = math.pi / (refine * k_max)
    return -x_m + step * np.arange(refine * n, dtype=np.float64), step


def extended_kernel(basis, kx, ky, eps_r, h, k0, beta_max, beta_p, height, green_fn=None):
    """I_M of Eq. 21 on real (kx, ky) (arrays of one shape): returns (I, gamma) with I of
    shape (M, M) + kx.shape, zero outside |k| <= beta_max."""
    kx = np.asarray(kx, dtype=np.float64)
    ky = np.asarray(ky, dtype=np.float64)
    br = np.hypot(kx, ky)
    bi = _contour.beta_imag(br, beta_p, height)
    slope = _contour.beta_imag_slope(br, beta_p, height)
    # gamma = beta_I / beta_R, continuous at the origin: 4 H / beta_p
    gamma = np.where(br > 0.0, bi / np.where(br > 0.0, br, 1.0), 4.0 * height / beta_p)
    kcx = kx * (1.0 + 1j * gamma)
    kcy = ky * (1.0 + 1j * gamma)
    hk = _reaction.kernel(basis, kcx, kcy, eps_r, h, k0, green_fn=green_fn)
    jac = (1.0 + 1j * slope) * (1.0 + 1j * gamma)
    inside = br <= beta_max
    return np.where(inside, hk * jac, 0.0), gamma


def monomials(order):
    """(a, b) with a + b <= order, by total degree."""
    return [(a, n - a) for n in range(order + 1) for a in range(n, -1, -1)]


def table(basis, eps_r, h, k0, beta_max, beta_p, height, n, order, refine=2, green_fn=None):
    """Z'_ab on the refined lattice (Eq. 24 with Appendix I and the zero-padded refinement).

    Returns (table of shape (M, M, refine n, refine n), spatial samples); axis -2 is dx,
    axis -1 is dy.
    """
    if n % 2:
        raise ValueError("n must be even (the Appendix I phase exp(-i pi N) is then 1)")
    k, dk = spectral_grid(n, beta_max)
    kx, ky = np.meshgrid(k, k, indexing="ij")
    im, gamma = extended_kernel(basis, kx, ky, eps_r, h, k0, beta_max, beta_p, height, green_fn)
    p = refine * n
    off = (p - n) // 2
    idx = np.arange(p)
    sign_in = (-1.0) ** (idx[:, None] + idx[None, :])       # (-1)^(n1' + n2') on the padded grid
    x, step = spatial_grid(n, beta_max, refine)
    sign_out = (-1.0) ** (idx[:, None] + idx[None, :])      # (-1)^(k1 + k2)
    kprime = dk * dk / (4.0 * math.pi ** 2) * sign_out
    gx, gy = gamma * kx, gamma * ky
    out = np.zeros(im.shape[:2] + (p, p), dtype=np.complex128)
    for a, b in monomials(order):
        spec = np.zeros(im.shape[:2] + (p, p), dtype=np.complex128)
        spec[..., off:off + n, off:off + n] = im * (gx ** a) * (gy ** b)
        f = kprime * np.fft.fft2(spec * sign_in, axes=(-2, -1))
        coef = (x[:, None] ** a) * (x[None, :] ** b) / (math.factorial(a) * math.factorial(b))
        out += coef * f
    return out, x


def direct_sum(basis, eps_r, h, k0, beta_max, beta_p, height, n, dx, dy, green_fn=None):
    """Eq. 21 by the rectangle rule with the exact contour factor E_I (no Taylor series, no
    FFT) at the points (dx, dy): the definition the table approximates."""
    k, dk = spectral_grid(n, beta_max)
    kx, ky = np.meshgrid(k, k, indexing="ij")
    im, gamma = extended_kernel(basis, kx, ky, eps_r, h, k0, beta_max, beta_p, height, green_fn)
    out = []
    for x, y in zip(np.atleast_1d(dx), np.atleast_1d(dy)):
        ph = np.exp(-1j * (kx * x + ky * y) + gamma * (kx * x + ky * y))
        out.append((im * ph).sum(axis=(-2, -1)) * dk * dk / (4.0 * math.pi ** 2))
    return np.moveaxis(np.array(out), 0, -1)


def interpolate(tab, x, dx, dy):
    """Second-order (three-point) Lagrange interpolation in dx and dy on the refined table
    (the end of Section III-B-3): nearest node and its two neighbours per axis."""
    step = x[1] - x[0]
    out = []
    for px, py in zip(np.atleast_1d(dx), np.atleast_1d(dy)):
        u = (px - x[0]) / step
        v = (py - x[0]) / step
        i0, j0 = int(round(u)), int(round(v))
        fu, fv = u - i0, v - j0
        wu = (0.5 * fu * (fu - 1.0), 1.0 - fu * fu, 0.5 * fu * (fu + 1.0))
        wv = (0.5 * fv * (fv - 1.0), 1.0 - fv * fv, 0.5 * fv * (fv + 1.0))
        acc = 0.0
        for s in range(3):
            for t in range(3):
                acc = acc + wu[s] * wv[t] * tab[..., i0 - 1 + s, j0 - 1 + t]
        out.append(acc)
    return np.moveaxis(np.array(out), 0, -1)
