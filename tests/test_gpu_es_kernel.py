"""The ES interpolation kernel of the FP32-mixed back-projection on the GPU (through the
C ABI): precorrected transform grid, tables against the oracle, errors.

- the grid the FFT stage leaves with the ES kernel is the exact sum of the precorrected
  samples, sum_j Y_j / phi_hat(omega_j) exp(-i beta_c,j s_k) (demodulated);
- ES (6 and 8 taps) and Lagrange (12 taps) tables against the oracle: 6 ES taps about as
  accurate as 12 Lagrange taps;
- the default FP32-mixed tabulation uses ES with 6 taps, FP64 Lagrange;
- ES requested where it cannot run (FP64, 12 taps) is an argument error.
"""
import os
import re

import numpy as np
import pytest

import workloads
from tests import cfft_cases as cc

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10}
CSRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "paper_1404_7357_gb300", "csrc")


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _phi_hat(om, w):
    """Fourier transform of the ES kernel of width w at complex omega (grid units), by a
    fine trapezoid rule on its definition (beta from the compiled tables' header)."""
    beta = float(re.search(r"kEsBeta%d = ([0-9.e+-]+);" % w, open(os.path.join(CSRC, "es_kernel.cuh")).read()).group(1))
    x = np.linspace(0.0, w / 2, 20001)
    t = 2 * x / w
    phi = np.exp(beta * (np.sqrt(np.maximum(0.0, 1 - t * t)) - 1))
    return 2.0 * np.trapezoid(phi[None, :] * np.cos(np.outer(om, x)), x, axis=1)


def test_precorrected_grid(torch_cuda):
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch("fp32", n=1024, n_rho=256, rho_max=4.0, q_max=2)
    ctx, _ = cc.gpu_table(wl, options={cfft.OPT_BP_KERNEL: 2})
    info = ctx.info()
    assert info["bp_kernel"] == 1 and info["bp_taps"] == 6
    nodes, hq = cc.oracle_harmonics(wl)
    grid = ctx.debug_buffer("grid").cpu().numpy()[0].astype(np.complex128)
    y = (hq[0] * (nodes["beta_c"] * nodes["weight"])).reshape(grid.shape[:-1] + (-1,))
    ds = info["delta_s"]
    om = (nodes["beta_c"] - wl.contour.beta_max / 2) * ds
    yp = y / _phi_hat(om, 6)
    k = np.arange(-info["grid_half"], info["grid_half"] + 1)
    sel = np.abs(k * ds) <= wl.rho_max
    gref = (yp @ np.exp(-1j * np.outer(nodes["beta_c"], k[sel] * ds))) * np.exp(1j * wl.contour.beta_max / 2 * k[sel] * ds)
    err = np.abs(grid[..., sel] - gref).max() / np.abs(gref).max()
    print("precorrected grid vs exact sum: %.3g" % err)
    assert err < 2e-5


def test_es_and_lagrange_against_oracle(torch_cuda):
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch("fp32", n=2048, n_rho=512, rho_max=8.0, q_max=4)
    ref, _, _ = cc.oracle_table(wl)
    errs = {}
    for name, opts in (("lagrange12", {cfft.OPT_BP_KERNEL: 1}), ("es6", {cfft.OPT_BP_KERNEL: 2}),
                       ("es8", {cfft.OPT_BP_KERNEL: 2, cfft.OPT_BP_TAPS: 8}), ("default", {})):
        ctx, got = cc.gpu_table(wl, options=opts)
        errs[name] = (cc.rel_err_per_pair(got, ref).max(), ctx.info()["bp_kernel"], ctx.info()["bp_taps"])
    print(errs)
    assert errs["default"][1:] == (1, 6)
    for name in errs:
        assert errs[name][0] < TOL["fp32"], name
    assert errs["es6"][0] < 1.5 * errs["lagrange12"][0]


def test_fp64_keeps_lagrange_and_es_errors(torch_cuda):
    from paper_1404_7357_gb300 import cfft
    wl = workloads.strip_fp64(n=1024, n_rho=128, rho_max=3.0, q_max=1)
    ctx, _ = cc.gpu_table(wl)
    assert ctx.info()["bp_kernel"] == 0 and ctx.info()["bp_taps"] == 16
    ctx = cc.gpu_context(wl, options={cfft.OPT_BP_KERNEL: 2})
    with pytest.raises(cfft.CfftError) as ei:
        ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP64, 1)
    assert ei.value.status == 1
    wl32 = cc.small_patch("fp32", n=1024, n_rho=128, rho_max=3.0, q_max=1)
    ctx = cc.gpu_context(wl32, options={cfft.OPT_BP_KERNEL: 2, cfft.OPT_BP_TAPS: 12})
    with pytest.raises(cfft.CfftError) as ei:
        ctx.tabulate_reactions(wl32.q_max, wl32.rho_max, wl32.n_rho, cfft.CFFT_FP32_MIXED, 1)
    assert ei.value.status == 1
