"""Error versus contour height and Taylor order: the study of the paper's Table I
(Section IV, "On the Contour height and Taylor's series order") with this library.

Two strip MBFs at the diagonal separation d = 21.2 lambda0 (Delta = (15, 15)
lambda0).  For each contour height, given as the paper's ratio gamma = beta_I /
beta_R near beta_R = 0 (here 4 H / beta_p for the parabolic contour), and each
fixed Taylor order 0..3, the FP64 GPU table (N = 4096 contour samples, rho to 25
lambda0 on 4096 points, |q| <= 4) is filled for the pair and compared with the
oracle's converged value (tests/golden/contour_study_strip.json, written by
make_contour_study.py from the oracle alone).  Errors in dB, 20 log10 |err| / |Z|.

The paper's numbers (its own MBFs, FFT2 of 2048^2) are context, not targets; the
trends are what the method implies: the error falls with the Taylor order, and a
contour that is too low (gamma = 1/400, below one node spacing here) leaves the
surface-wave poles visible to the rectangle rule, so that more Taylor terms stop
helping.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads
from tests import cfft_cases as cc

pytestmark = pytest.mark.gpu

GAMMAS = (1 / 50, 1 / 100, 1 / 130, 1 / 200, 1 / 400)
ORDERS = (0, 1, 2, 3)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _ref():
    with open(os.path.join(os.path.dirname(__file__), "golden", "contour_study_strip.json")) as f:
        d = json.load(f)
    return complex(d["reference"]["z_re"], d["reference"]["z_im"]), d["meta"]


def test_contour_height_and_taylor_order(torch_cuda):
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    zref, meta = _ref()
    pos = torch.tensor([[0.0, 0.0], [meta["dx"], meta["dy"]]], dtype=torch.float64, device="cuda:0")
    table = {}
    for gamma in GAMMAS:
        for order in ORDERS:
            wl = workloads.strip_fp64(n=4096, n_rho=4096, rho_max=25.0, q_max=4)
            c = wl.contour
            ctx = cfft.Context(0)
            s = wl.substrate
            ctx.set_substrate(s.eps_r, s.h, s.k0)
            ctx.set_mbf_spectra_strip(wl.element.length, wl.element.strip_width)
            ctx.build_contour(c.n, c.beta_max, c.beta_p, gamma * c.beta_p / 4.0, order)
            ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP64, 1)
            z = torch.empty((2, 2), dtype=torch.complex128, device="cuda:0")
            ctx.fill_reduced_matrix(pos, None, z)
            got = complex(z[1, 0].item())
            table[(gamma, order)] = 20.0 * math.log10(abs(got - zref) / abs(zref))
    print("\nerror (dB) vs contour height and Taylor order, d = %.1f lambda0" % meta["rho"])
    print("order / gamma " + " ".join("%8s" % ("1/%d" % round(1 / g)) for g in GAMMAS))
    for order in ORDERS:
        print("%13d " % order + " ".join("%8.1f" % table[(g, order)] for g in GAMMAS))
    # the error falls with the Taylor order for the moderate heights
    for gamma in (1 / 100, 1 / 130, 1 / 200):
        errs = [table[(gamma, o)] for o in ORDERS]
        assert all(b < a for a, b in zip(errs, errs[1:])), (gamma, errs)
    # the recommended range (gamma 1/100 .. 1/200) with 3 terms beats the too-low contour
    best_mid = min(table[(g, 3)] for g in (1 / 100, 1 / 130, 1 / 200))
    assert best_mid < min(table[(1 / 400, o)] for o in ORDERS)
