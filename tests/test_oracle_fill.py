"""Pin for the oracle's exact reduced-matrix fill.

A small array of elements that each carry two Gaussian currents (one MBF
each, Q = I; the first along x, the second along y) under a unit dyadic has a
closed-form reduced matrix: an element rotated by theta carries its current a
at R(theta) c_a along R(theta) d_a, so
Z'[(m,a),(n,b)] = (R(theta_m) d_a . R(theta_n) d_b) exp(-|D|^2 / 8 s^2) / (8 pi s^2),
D = r_m - r_n + R(theta_m) c_a - R(theta_n) c_b.  This pins the pair geometry
(Delta = r_test - r_basis, phi), the block layout and the rotation classes:
with one x- and one y-directed current the two mixed classes (0, 90) and
(90, 0) give different, non-zero blocks, so exchanging them is caught.
"""
import math

import numpy as np

from oracle import contour, fill, green, reaction, spectra

K0 = 2 * math.pi


def test_gaussian_array_closed_form():
    s = 0.1
    cs = np.array([[0.04, -0.02], [-0.03, 0.05]])
    dirs = np.array([[1.0, 0.0], [0.0, 1.0]])          # current a along dirs[a]
    bs = spectra.BasisSet("gaussian", np.eye(2), cx=cs[:, 0], cy=cs[:, 1],
                          direction=np.array([0, 1]), s=s)
    pos = np.array([[0.0, 0.0], [0.25, 0.1], [-0.12, 0.3]])
    rot = np.array([0, 1, 0])
    qs = np.arange(-16, 17)
    mats = []
    for n in (2000, 4000):                 # beta_p = 12 is a cell boundary of both
        c = contour.contour_nodes(n, 60.0, 12.0, 0.4)
        hq = {cls: reaction.harmonics(bs, c["beta_c"], qs, 96, 0, 0, K0,
                                      *reaction.rotation_angles(cls),
                                      green_fn=green.identity_green)
              for cls in range(4)}
        mats.append(fill.full_matrix(hq, qs, c["beta_c"], c["weight"], pos, rot))
    z = (4 * mats[1] - mats[0]) / 3

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
                    exact[2 * m + a, 2 * n + b] = (align * math.exp(-d @ d / (8 * s * s))
                                                   / (8 * math.pi * s * s))
    scale = 1 / (8 * math.pi * s * s)
    assert np.abs(z - exact).max() < 1e-9 * scale
