"""Pins for the oracle's reduced MBF system (Section II, Eqs. 1-4).

- With as many MBFs as basis functions (Q square and invertible) the reduced
  system is the full system in another basis: the expanded reduced solution equals
  the full MoM solution, for every antenna and basis function.
- With fewer MBFs the reduced solution is the Galerkin projection: the full
  residual Z (Q I') - V is orthogonal to every MBF of every antenna.
- The spectral MBF reaction (Eq. 9 with the MBF spectra of Eq. 11, as ``fill``
  evaluates it) equals Q^H Z Q of Eq. 3 built from the elementary reactions
  (the same spectral integral with one basis function per column): this ties the
  conjugation of Eq. 11 to the Hermitian transpose of Eq. 3.
- A transpose in place of the Hermitian transpose is caught.
"""
import math

import numpy as np

from oracle import contour, fill, reaction, solve, spectra

K0 = 2 * math.pi


def _system(seed, a=3, b=5):
    rng = np.random.default_rng(seed)
    zb = rng.standard_normal((a, a, b, b)) + 1j * rng.standard_normal((a, a, b, b))
    for m in range(a):                       # diagonally dominant self blocks: well conditioned
        zb[m, m] += 6.0 * np.eye(b)
    v = rng.standard_normal((a, b)) + 1j * rng.standard_normal((a, b))
    return zb, v


def _full(zb):
    a, _, b, _ = zb.shape
    return zb.transpose(0, 2, 1, 3).reshape(a * b, a * b)


def test_square_q_reproduces_the_full_solution():
    zb, v = _system(1)
    rng = np.random.default_rng(2)
    b = zb.shape[2]
    q = rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b))
    ip = solve.solve_reduced(solve.reduced_matrix(q, zb), solve.reduced_excitation(q, v))
    i_red = solve.expand_currents(q, ip)
    i_full = np.linalg.solve(_full(zb), v.reshape(-1)).reshape(v.shape)
    assert np.abs(i_red - i_full).max() < 1e-10 * np.abs(i_full).max()
    # a delta-gap port: the port current is the full solution's current there
    amps = np.array([1.0, 0.5j, -0.7])
    vport = np.zeros_like(v)
    vport[:, 2] = amps
    ip = solve.solve_reduced(solve.reduced_matrix(q, zb), solve.port_excitation(q, 2, amps))
    i_full = np.linalg.solve(_full(zb), vport.reshape(-1)).reshape(v.shape)
    assert np.abs(solve.port_currents(q, 2, ip) - i_full[:, 2]).max() < 1e-10 * np.abs(i_full).max()


def test_fewer_mbfs_give_the_galerkin_projection():
    zb, v = _system(3)
    rng = np.random.default_rng(4)
    q = rng.standard_normal((5, 2)) + 1j * rng.standard_normal((5, 2))
    ip = solve.solve_reduced(solve.reduced_matrix(q, zb), solve.reduced_excitation(q, v))
    i = solve.expand_currents(q, ip)
    resid = (_full(zb) @ i.reshape(-1) - v.reshape(-1)).reshape(v.shape)
    proj = resid @ np.conj(q)                      # Q^H r_m for every antenna
    assert np.abs(proj).max() < 1e-11 * np.abs(v).max()
    assert np.abs(resid).max() > 1e-3 * np.abs(v).max()     # the projection is not the solution


def test_transpose_instead_of_hermitian_is_caught():
    zb, v = _system(5)
    rng = np.random.default_rng(6)
    q = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    zr = np.einsum("ia,mnij,jb->manb", q, zb, q).reshape(15, 15)      # Q^T Z Q
    vr = (v @ q).reshape(-1)                                           # Q^T V
    i_red = solve.expand_currents(q, solve.solve_reduced(zr, vr))
    i_full = np.linalg.solve(_full(zb), v.reshape(-1)).reshape(v.shape)
    # Q^T is also invertible, so Q^T Z Q reproduces the full solution too: the slip only
    # shows once the reduced matrix comes from the spectral MBF reaction (next test)
    assert np.abs(i_red - i_full).max() < 1e-9 * np.abs(i_full).max()
    mixed = solve.solve_reduced(solve.reduced_matrix(q, zb), vr)        # Q^H Z Q with Q^T V
    assert np.abs(solve.expand_currents(q, mixed) - i_full).max() > 1e-2 * np.abs(i_full).max()


def test_spectral_mbf_reaction_equals_q_hermitian_z_q():
    rng = np.random.default_rng(8)
    cx = np.array([-0.08, 0.0, 0.07, -0.03, 0.05])
    cy = np.array([0.02, -0.06, 0.0, 0.08, -0.04])
    d = np.array([0, 0, 0, 1, 1])
    geom = dict(cx=cx, cy=cy, direction=d, half_len=np.full(5, 0.05), width=np.full(5, 0.03))
    q = rng.standard_normal((5, 2)) + 1j * rng.standard_normal((5, 2))
    eps_r, h = 4.4, 0.03
    kd = K0 * math.sqrt(eps_r)
    c = contour.contour_nodes(400, 5 * kd, 1.3 * kd, 6 * 5 * kd / 400)
    qs = np.arange(-6, 7)
    pos = np.array([[0.0, 0.0], [0.9, 0.4]])
    rot = np.zeros(2, dtype=int)
    pairs = [(0, 0), (0, 1), (1, 0)]
    mbf = spectra.BasisSet("rooftop", q, **geom)
    elem = spectra.BasisSet("rooftop", np.eye(5), **geom)          # one basis function per column
    hq_m = reaction.harmonics(mbf, c["beta_c"], qs, 64, eps_r, h, K0)
    hq_e = reaction.harmonics(elem, c["beta_c"], qs, 64, eps_r, h, K0)
    zm = fill.entries({0: hq_m}, qs, c["beta_c"], c["weight"], pos, rot, pairs)   # (pairs, 2, 2)
    ze = fill.entries({0: hq_e}, qs, c["beta_c"], c["weight"], pos, rot, pairs)   # (pairs, 5, 5)
    for k in range(len(pairs)):
        eq3 = np.conj(q).T @ ze[k] @ q
        assert np.abs(zm[k] - eq3).max() < 1e-12 * np.abs(eq3).max()
    # with Q^T in place of Q^H the relation breaks
    assert np.abs(zm[1] - q.T @ ze[1] @ q).max() > 1e-2 * np.abs(zm[1]).max()
