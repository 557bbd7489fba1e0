"""Reduced MBF system: excitation, solution and port currents (Section II, Eqs. 1-4).

With the MBFs of every antenna in the columns of Q (B elementary basis functions by
M MBFs, the same Q for identical antennas), the currents of antenna m are
I_m = Q I'_m, the reduced matrix blocks are Z'_mn = Q^H Z_mn Q (Eq. 3) -- which
``fill`` evaluates spectrally -- and the reduced excitation is V'_m = Q^H V_m
(Eq. 4).  The reduced system Z' I' = V' is solved directly (the paper notes that
the reduction makes direct inversion affordable); a library LU is the step here.

For a delta-gap port across elementary basis function p of every antenna, driven
by voltage a_m, V_m = a_m e_p, so V'_m = a_m conj(Q[p, :]) and the port current is
(Q I'_m)[p]; the active input impedance is a_m / I_port,m.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np


def reduced_excitation(q, v):
    """V' = Q^H V_m per antenna: q (B, M), v (A, B) -> (A * M,) in the row order of Z'."""
    q = np.asarray(q, dtype=np.complex128)
    v = np.asarray(v, dtype=np.complex128)
    return (v @ np.conj(q)).reshape(-1)          # row m: sum_i conj(Q_ia) V_m,i


def port_excitation(q, port, amplitudes):
    """V' for a delta-gap port across basis function `port` of every antenna."""
    q = np.asarray(q, dtype=np.complex128)
    a = np.asarray(amplitudes, dtype=np.complex128)
    v = np.zeros((a.size, q.shape[0]), dtype=np.complex128)
    v[:, port] = a
    return reduced_excitation(q, v)


def solve_reduced(zp, vp):
    """I' with Z' I' = V' (dense LU of the library)."""
    return np.linalg.solve(np.asarray(zp, dtype=np.complex128), np.asarray(vp, dtype=np.complex128))


def expand_currents(q, ip):
    """Elementary-basis currents I_m = Q I'_m: ip (A * M,) -> (A, B)."""
    q = np.asarray(q, dtype=np.complex128)
    m = q.shape[1]
    return np.asarray(ip, dtype=np.complex128).reshape(-1, m) @ q.T


def port_currents(q, port, ip):
    """Current through the port basis function of every antenna: (Q I'_m)[port]."""
    return expand_currents(q, ip)[:, port]


def reduced_matrix(q, z_blocks):
    """Z' from elementary blocks (Eq. 3): z_blocks (A, A, B, B) -> (A * M, A * M).
    (The spectral fill computes Z' directly; this form serves checks on small cases.)"""
    q = np.asarray(q, dtype=np.complex128)
    zb = np.asarray(z_blocks, dtype=np.complex128)
    a, m = zb.shape[0], q.shape[1]
    zr = np.einsum("ia,mnij,jb->manb", np.conj(q), zb, q)
    return zr.reshape(a * m, a * m)
