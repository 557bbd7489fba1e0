"""Exact per-entry reduced matrix Z' of an array of identical elements.

Eq. 3 gives the reduced block Z'_mn = Q^H Z_mn Q of test element m and basis
element n; Eq. 9 evaluates it spectrally for the relative position
Delta = r_m - r_n = rho (cos phi, sin phi).  Through the harmonic form
(see ``reaction``) each entry is

  Z'[(m, a), (n, b)] = sum_q exp(i q phi) Z^{cls}_ab,q(rho)

with Z_ab,q(rho) evaluated here at the exact rho by the matched-contour Bessel
sum (no table, no interpolation).  ``cls`` is the rotation class of the pair
(element rotations in {0, 90 deg}).  For m = n (self block) the same formula at
rho = 0 is used: only q = 0 survives since J_q(0) = 0 for q != 0.  (The paper
computes self blocks once with the traditional MBF method, Section IV-E; here
they come from the same spectral integral.)

Row/column layout: row index m*M + a, column index n*M + b.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np

from . import reaction as _reaction


def pair_geometry(pos, m, n):
    """(rho, phi) of Delta = r_m - r_n."""
    d = np.asarray(pos[m], dtype=np.float64) - np.asarray(pos[n], dtype=np.float64)
    return float(np.hypot(d[0], d[1])), float(np.arctan2(d[1], d[0]))


def class_index(rot, m, n):
    """Rotation class of (test m, basis n) with rotations in {0, 1} (0 or 90 deg)."""
    return 2 * int(rot[m]) + int(rot[n])


def entries(hq_by_class, qs, beta_c, weight, pos, rot, pairs):
    """Exact reduced-matrix blocks for the listed element pairs.

    hq_by_class: dict cls -> (M, M, nq, n) harmonics on the contour nodes.
    pairs: iterable of (m, n).  Returns array (len(pairs), M, M).
    """
    out = []
    for m, n in pairs:
        rho, phi = pair_geometry(pos, m, n)
        hq = hq_by_class[class_index(rot, m, n)]
        zq = _reaction.table_bessel(hq, qs, beta_c, weight, np.array([rho]))[..., 0]
        out.append(_reaction.reaction_from_table(zq, qs, phi))
    return np.array(out)


def full_matrix(hq_by_class, qs, beta_c, weight, pos, rot):
    """Dense (A*M, A*M) reduced matrix for a small array."""
    a_count = len(pos)
    m_count = next(iter(hq_by_class.values())).shape[0]
    pairs = [(m, n) for m in range(a_count) for n in range(a_count)]
    blocks = entries(hq_by_class, qs, beta_c, weight, pos, rot, pairs)
    z = np.empty((a_count * m_count, a_count * m_count), dtype=np.complex128)
    for (m, n), blk in zip(pairs, blocks):
        z[m * m_count:(m + 1) * m_count, n * m_count:(n + 1) * m_count] = blk
    return z
