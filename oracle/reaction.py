"""MBF reaction tables by direct quadrature of Eq. 9 (FP64 definition).

Definitions (Section III-A, Eqs. 7-11), with Delta = r_test - r_basis =
rho (cos phi, sin phi) and k = beta (cos alpha, sin alpha):

  H_ab(k)     = M_a(k)^T . G(k) . Mbar_b(k)                          (Eq. 10)
  Z'_ab       = 1/(4 pi^2) int int H_ab(k) exp(-i k.Delta) beta d beta d alpha
                along the deformed contour beta = beta_c(beta_R)      (Eq. 9)

Expanding H_ab in azimuthal harmonics and integrating over alpha with the
Jacobi-Anger identity gives the harmonic reaction table

  H_ab,q(beta) = 1/(2 pi) int_0^{2 pi} H_ab(beta, alpha) exp(-i q alpha) d alpha
  Z_ab,q(rho)  = (-i)^q / (2 pi) int_C H_ab,q(beta) J_q(beta rho) beta d beta
  Z'_ab(rho, phi) = sum_q Z_ab,q(rho) exp(i q phi)

and, equivalently, the alpha form used by a one-dimensional FFT in beta,

  g_ab,q(s)   = int_C H_ab,q(beta) beta exp(-i beta s) d beta
  Z_ab,q(rho) = 1/(4 pi^2) int_0^{2 pi} exp(i q alpha) g_ab,q(rho cos alpha) d alpha
              = 1/(2 pi^2) int_0^{pi} cos(q alpha) g_ab,q(rho cos alpha) d alpha.

Quadratures here:
  * ``harmonics``     -- trapezoid rule in alpha with n_alpha points (exact up
                         to aliasing of harmonics >= n_alpha - |q|).
  * ``table_bessel``  -- "O2 matched": the contour rectangle rule of Eq. 8/23
                         with the caller's nodes and weights, Bessel functions of
                         complex argument from scipy (a library routine).
  * ``table_alpha``   -- the same beta nodes with exact exponentials and a
                         midpoint rule in alpha (cross-check of O2).
  * ``table_adaptive``-- "O1 converged": adaptive Gauss-Kronrod along the
                         contour (the truncated integral itself).

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np
import scipy.special as sp
import scipy.integrate as si

from . import green as _green
from . import spectra as _spectra


def kernel(basis, kx, ky, eps_r, h, k0, theta_t=0.0, theta_b=0.0, green_fn=None):
    """H_ab(k) of Eq. 10 for all MBF pairs: array (M, M) + broadcast shape.

    Test MBFs on an element rotated by theta_t, basis MBFs on one rotated by theta_b.
    green_fn defaults to the grounded slab; oracle.green.identity_green isolates
    the transform from the substrate in tests.
    """
    green_fn = green_fn or _green.dyadic_green
    gxx, gxy, gyy = green_fn(kx, ky, eps_r, h, k0)
    tx, ty = _spectra.mbf_spectra(basis, kx, ky, theta=theta_t, conjugate_side=False)
    bx, by = _spectra.mbf_spectra(basis, kx, ky, theta=theta_b, conjugate_side=True)
    # sum over u, v in {x, y} of M_a,u G_uv Mbar_b,v
    gx = gxx * bx + gxy * by     # (G . Mbar_b)_x, shape (M, ...)
    gy = gxy * bx + gyy * by     # (G . Mbar_b)_y
    return tx[:, None] * gx[None, :] + ty[:, None] * gy[None, :]


def _harmonics_slice(args):
    return harmonics(*args)


def harmonics(basis, beta, qs, n_alpha, eps_r, h, k0, theta_t=0.0, theta_b=0.0,
              green_fn=None, chunk=256, workers=None):
    """H_ab,q(beta_j) by the n_alpha-point trapezoid rule in alpha.

    beta: complex array (n,).  Returns (M, M, len(qs), n) complex128.
    workers > 1 splits the nodes over that many spawned processes (each node is
    independent; the arithmetic per node is unchanged).
    """
    beta = np.asarray(beta, dtype=np.complex128)
    qs = np.asarray(qs)
    if workers and workers > 1 and beta.size > 4 * chunk:
        import concurrent.futures as cf
        import multiprocessing as mp
        import os
        parts = np.array_split(beta, workers * 4)
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
        try:
            with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
                res = list(ex.map(_harmonics_slice,
                                  [(basis, p, qs, n_alpha, eps_r, h, k0, theta_t, theta_b,
                                    green_fn, chunk, None) for p in parts]))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        return np.concatenate(res, axis=-1)
    alpha = 2.0 * np.pi * np.arange(n_alpha) / n_alpha
    ca, sa = np.cos(alpha), np.sin(alpha)
    dft = np.exp(-1j * np.outer(alpha, qs)) / n_alpha          # (n_alpha, nq)
    m = basis.n_mbf
    out = np.empty((m, m, len(qs), beta.size), dtype=np.complex128)
    for j0 in range(0, beta.size, chunk):
        b = beta[j0:j0 + chunk]
        kx = b[:, None] * ca[None, :]
        ky = b[:, None] * sa[None, :]
        hk = kernel(basis, kx, ky, eps_r, h, k0, theta_t, theta_b, green_fn)  # (M,M,nb,na)
        out[:, :, :, j0:j0 + chunk] = np.moveaxis(hk @ dft, -1, 2)
    return out


def _sign_pow(q):
    return (-1.0) ** (int(q) % 2)


def bessel_jq(q, z):
    """J_q(z) for integer q of either sign, complex z (scipy's jv)."""
    q = int(q)
    if q >= 0:
        return sp.jv(q, z)
    return _sign_pow(q) * sp.jv(-q, z)


def table_bessel(hq, qs, beta_c, weight, rho):
    """O2 (matched contour): Z_q(rho_r) = (-i)^q/(2 pi) sum_j w_j beta_j H_q(beta_j) J_q(beta_j rho_r).

    hq: (..., nq, n) harmonics at the contour nodes; returns (..., nq, nrho).
    """
    rho = np.asarray(rho, dtype=np.float64)
    x = hq * (weight * beta_c)
    out = np.empty(hq.shape[:-1] + (rho.size,), dtype=np.complex128)
    for iq, q in enumerate(qs):
        jmat = bessel_jq(q, np.outer(beta_c, rho))               # (n, nrho)
        out[..., iq, :] = ((-1j) ** int(q) / (2.0 * np.pi)) * (x[..., iq, :] @ jmat)
    return out


def alpha_nodes(rho, beta_abs_max, q_abs_max, margin=40):
    """Midpoint count for the alpha form: the integrand's alpha content reaches
    |beta| rho; the rule resolves it with 2 N' > |beta| rho + |q| + margin."""
    z = beta_abs_max * rho
    return int(np.ceil((z + q_abs_max + margin + 4.0 * np.cbrt(z)) / 2.0)) + 1


def table_alpha(hq, qs, beta_c, weight, rho, n_alpha_prime=None):
    """Alpha form with exact exponentials: 1/(2 pi^2) (pi/N') sum_l cos(q a_l) g_q(rho cos a_l).

    g_q(s) = sum_j w_j beta_j H_q(beta_j) exp(-i beta_j s) is evaluated exactly.
    """
    rho = np.asarray(rho, dtype=np.float64)
    x = hq * (weight * beta_c)
    out = np.empty(hq.shape[:-1] + (rho.size,), dtype=np.complex128)
    bmax = np.abs(beta_c).max()
    qmax = int(np.max(np.abs(qs)))
    for ir, r in enumerate(rho):
        npr = n_alpha_prime or alpha_nodes(r, bmax, qmax)
        a = (np.arange(npr) + 0.5) * np.pi / npr
        s = r * np.cos(a)
        e = np.exp(-1j * np.outer(beta_c, s))                    # (n, npr)
        g = x @ e                                                # (..., nq, npr)
        c = np.cos(np.outer(np.asarray(qs, dtype=np.float64), a))  # (nq, npr)
        out[..., ir] = (g * c).sum(-1) * (1.0 / (2.0 * np.pi ** 2)) * (np.pi / npr)
    return out


def harmonic_at(basis, a, b, q, beta, n_alpha, eps_r, h, k0, theta_t=0.0, theta_b=0.0,
                green_fn=None):
    """H_ab,q at a single complex beta (for adaptive quadrature)."""
    return harmonics(basis, np.array([beta]), [q], n_alpha, eps_r, h, k0, theta_t, theta_b,
                     green_fn)[a, b, 0, 0]


def table_adaptive(basis, a, b, q, rho, beta_max, beta_p, height, n_alpha, eps_r, h, k0,
                   theta_t=0.0, theta_b=0.0, green_fn=None, breakpoints=(), epsabs=1e-13,
                   epsrel=1e-11, limit=400):
    """O1 (converged): adaptive Gauss-Kronrod of Eq. 9's harmonic form along the contour."""
    from .contour import contour_point

    def integrand(t):
        bc, dbc = contour_point(t, beta_p, height)
        bc = complex(bc)
        hq = harmonic_at(basis, a, b, q, bc, n_alpha, eps_r, h, k0, theta_t, theta_b, green_fn)
        return hq * bessel_jq(q, bc * rho) * bc * complex(dbc)

    pts = sorted({p for p in list(breakpoints) + [beta_p, k0] if 0.0 < p < beta_max})
    re = si.quad(lambda t: integrand(t).real, 0.0, beta_max, points=pts or None,
                 epsabs=epsabs, epsrel=epsrel, limit=limit)[0]
    im = si.quad(lambda t: integrand(t).imag, 0.0, beta_max, points=pts or None,
                 epsabs=epsabs, epsrel=epsrel, limit=limit)[0]
    return ((-1j) ** int(q) / (2.0 * np.pi)) * (re + 1j * im)


def reaction_from_table(zq, qs, phi):
    """Z'(rho, phi) = sum_q Z_q(rho) exp(i q phi); zq (..., nq), phi broadcastable."""
    qs = np.asarray(qs, dtype=np.float64)
    return (zq * np.exp(1j * np.multiply.outer(phi, qs))).sum(-1)


def rotation_angles(cls):
    """Rotation class index -> (theta_test, theta_basis) in radians.

    Class 0 = (0, 0), 1 = (0, 90 deg), 2 = (90 deg, 0), 3 = (90 deg, 90 deg).
    """
    half_pi = np.pi / 2.0
    return [(0.0, 0.0), (0.0, half_pi), (half_pi, 0.0), (half_pi, half_pi)][cls]
