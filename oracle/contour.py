"""Parabolic contour in the complex radial wavenumber plane (Eq. 8, Fig. 1).

The radial spectral variable of Eq. 7 is deformed to beta_c = beta_R + i beta_I
(Eq. 8) while the integration runs along the real part beta_R.  The paper names
a parabolic deformation (Fig. 1 caption, Section III-A) and integrates with the
rectangle rule (Section III-B-3, Eq. 23).  Reading used here: a parabola of peak
height ``height`` on [0, beta_p] that returns to the real axis at beta_p (beyond
all surface-wave poles), the real axis beyond beta_p, truncated at beta_max
(5 k_d, Section III-A), sampled at midpoints beta_R = (j + 1/2) h.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np


def beta_imag(beta_r, beta_p, height):
    """Imaginary part of the contour, 4 H b (b_p - b) / b_p^2 on [0, b_p], else 0."""
    beta_r = np.asarray(beta_r, dtype=np.float64)
    inside = (beta_r >= 0.0) & (beta_r < beta_p)
    return np.where(inside, 4.0 * height * beta_r * (beta_p - beta_r) / beta_p ** 2, 0.0)


def beta_imag_slope(beta_r, beta_p, height):
    """d beta_I / d beta_R, the slope entering the Jacobian (1 + i d beta_I/d beta_R) of Eq. 8."""
    beta_r = np.asarray(beta_r, dtype=np.float64)
    inside = (beta_r >= 0.0) & (beta_r < beta_p)
    return np.where(inside, 4.0 * height * (beta_p - 2.0 * beta_r) / beta_p ** 2, 0.0)


def contour_nodes(n, beta_max, beta_p, height):
    """Rectangle-rule nodes of the deformed contour.

    Returns a dict with, for j = 0..n-1:
      beta_r  = (j + 1/2) h,  h = beta_max / n
      beta_i  = beta_I(beta_r)
      beta_c  = beta_r + i beta_i                 (Eq. 8)
      weight  = h (1 + i d beta_I / d beta_R)     (Eq. 8 Jacobian times d beta_R)
    """
    h = beta_max / n
    beta_r = (np.arange(n, dtype=np.float64) + 0.5) * h
    beta_i = beta_imag(beta_r, beta_p, height)
    slope = beta_imag_slope(beta_r, beta_p, height)
    return {
        "h": h,
        "beta_r": beta_r,
        "beta_i": beta_i,
        "beta_c": beta_r + 1j * beta_i,
        "weight": h * (1.0 + 1j * slope),
    }


def contour_point(t, beta_p, height):
    """beta_c(t) and d beta_c / dt for a real parameter t = beta_R (for adaptive quadrature)."""
    return (t + 1j * beta_imag(t, beta_p, height),
            1.0 + 1j * beta_imag_slope(t, beta_p, height))
