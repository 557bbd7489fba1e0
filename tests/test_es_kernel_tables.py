"""The ES interpolation kernel tables compiled into the FP32-mixed back-projection
(csrc/es_kernel.cuh), checked on the CPU against the kernel's definition
phi(x) = exp(beta (sqrt(1 - (2x/w)^2) - 1)), |x| <= w/2:

- the per-tap polynomials reproduce phi at every offset of every tap;
- the Gauss-Legendre rule of the Fourier transform reproduces phi_hat(omega) of a direct
  fine quadrature, at real and complex omega;
- with those tables, precorrected samples of a band-limited signal at sigma = 4 are
  interpolated to the stated accuracy (2e-6 for w = 6; 1e-8 for w = 8, plus the float32
  rounding of the tables);
- the header is what its generator writes.
"""
import os
import re
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1404_7357_gb300", "csrc")


def _tables():
    text = open(os.path.join(CSRC, "es_kernel.cuh")).read()
    out = {}
    for w in (6, 8):
        beta = float(re.search(r"kEsBeta%d = ([0-9.e+-]+);" % w, text).group(1))
        body = re.search(r"kEsPoly%d\[%d\]\[(\d+)\] = \{(.*?)\};" % (w, w), text, re.S)
        rows = [np.array([float(v.rstrip("f")) for v in r.split(",") if v.strip()])
                for r in re.findall(r"\{([^{}]*)\}", body.group(2))]
        qx = np.array([float(v.rstrip("f")) for v in
                       re.search(r"kEsQuadX%d\[\d+\] = \{(.*?)\};" % w, text, re.S).group(1).split(",")])
        qw = np.array([float(v.rstrip("f")) for v in
                       re.search(r"kEsQuadW%d\[\d+\] = \{(.*?)\};" % w, text, re.S).group(1).split(",")])
        out[w] = (beta, np.array(rows), qx, qw)
    return out


def _phi(x, w, beta):
    t = 2.0 * np.asarray(x) / w
    return np.where(np.abs(t) <= 1.0, np.exp(beta * (np.sqrt(np.maximum(0.0, 1.0 - t * t)) - 1.0)), 0.0)


def _phi_hat_fine(om, w, beta):
    x = np.linspace(0.0, w / 2, 200001)
    f = _phi(x, w, beta)[None, :] * np.cos(np.outer(om, x))
    return 2.0 * np.trapezoid(f, x, axis=1)


@pytest.mark.parametrize("w", [6, 8])
def test_tap_polynomials_reproduce_the_kernel(w):
    beta, polys, _, _ = _tables()[w]
    half = w // 2 - 1
    f = np.linspace(0.0, 1.0, 1001)
    err = 0.0
    for m in range(w):
        val = np.polynomial.polynomial.polyval(f, polys[m])
        err = max(err, np.abs(val - _phi(f + half - m, w, beta)).max())
    print("w", w, "max |poly - phi|", err)
    assert err < 3e-7


@pytest.mark.parametrize("w", [6, 8])
def test_fourier_quadrature(w):
    beta, _, qx, qw = _tables()[w]
    om = np.linspace(-np.pi / 4, np.pi / 4, 9)
    quad = 2.0 * (qw[None, :] * np.cos(np.outer(om, qx))).sum(1)
    fine = _phi_hat_fine(om, w, beta)
    assert np.abs(quad / fine - 1).max() < 1e-6
    # complex omega: cos((a + i b) x) = cos(a x) cosh(b x) - i sin(a x) sinh(b x)
    a, b = 0.5, 0.05
    quad_c = 2.0 * (qw * (np.cos(a * qx) * np.cosh(b * qx) - 1j * np.sin(a * qx) * np.sinh(b * qx))).sum()
    x = np.linspace(0.0, w / 2, 200001)
    fine_c = 2.0 * np.trapezoid(_phi(x, w, beta) * np.cos((a + 1j * b) * x), x)
    assert abs(quad_c / fine_c - 1) < 1e-6


# aliasing bound of the kernel (2e-6, 1e-8) plus its float32 polynomial tables (~1e-8)
@pytest.mark.parametrize("w,bound", [(6, 2e-6), (8, 3e-8)])
def test_precorrected_interpolation_accuracy(w, bound):
    """Sum of tones e^{-i omega_j k} with |omega_j| <= pi/4 (sigma = 4) and random
    amplitudes: samples divided by phi_hat(omega_j), interpolated with the tables' kernel
    at random u, against the exact sum."""
    beta, polys, qx, qw = _tables()[w]
    rng = np.random.default_rng(5)
    om = rng.uniform(-np.pi / 4, np.pi / 4, 64) + 1j * rng.uniform(0, 2e-3, 64)
    amp = rng.normal(size=64) + 1j * rng.normal(size=64)
    ph = 2.0 * (qw[None, :] * (np.cos(np.outer(om.real, qx)) * np.cosh(np.outer(om.imag, qx))
                               - 1j * np.sin(np.outer(om.real, qx)) * np.sinh(np.outer(om.imag, qx)))).sum(1)
    k = np.arange(-40, 41)
    grid = (amp / ph) @ np.exp(-1j * np.outer(om, k))
    half = w // 2 - 1
    err = 0.0
    scale = np.abs(amp).sum()
    for u in rng.uniform(-20, 20, 200):
        fl = int(np.floor(u))
        f = u - fl
        taps = fl - half + np.arange(w)
        wts = np.array([np.polynomial.polynomial.polyval(f, polys[m]) for m in range(w)])
        val = (grid[taps + 40] * wts).sum()
        err = max(err, abs(val - (amp * np.exp(-1j * om * u)).sum()) / scale)
    print("w", w, "interpolation error / sum |amp|", err)
    assert err < bound


def test_header_matches_generator(tmp_path):
    import shutil
    shutil.copy(os.path.join(CSRC, "gen_es_kernel.py"), tmp_path / "gen_es_kernel.py")
    subprocess.run([sys.executable, str(tmp_path / "gen_es_kernel.py")], check=True, capture_output=True)
    assert (tmp_path / "es_kernel.cuh").read_text() == open(os.path.join(CSRC, "es_kernel.cuh")).read()
