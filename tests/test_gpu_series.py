"""The two series of the contour factor exp(beta_I s) that split the transform into FFTs
(Section III-B-3, Eq. 22): the paper's Taylor series and its Chebyshev form about the
middle of beta_I / H (cfft_set_option CONTOUR_SERIES), through the C ABI.

- both against the exact exponential sum on the transform grid (the definition the
  series approximate) and the whole table against the oracle, FP64 and FP32-mixed;
- the Chebyshev form needs fewer FFTs for the same remainder bound (the automatic
  choice takes it when it does), and its error falls with its degree;
- an explicit Taylor order keeps the paper's series.
"""
import numpy as np
import pytest

import workloads
from tests import cfft_cases as cc

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _grid_error(ctx, wl):
    """Transform grid against sum_j Y_j exp(-i beta_c,j s_k), demodulated, |s_k| <= rho_max."""
    nodes, hq = cc.oracle_harmonics(wl)
    info = ctx.info()
    grid = ctx.debug_buffer("grid").cpu().numpy()[0].astype(np.complex128)
    yref = (hq[0] * (nodes["beta_c"] * nodes["weight"])).reshape(grid.shape[:-1] + (-1,))
    k = np.arange(-info["grid_half"], info["grid_half"] + 1)
    s = k * info["delta_s"]
    sel = np.abs(s) <= wl.rho_max
    e = np.exp(-1j * np.outer(nodes["beta_c"], s[sel]))
    gref = (yref @ e) * np.exp(1j * wl.contour.beta_max / 2 * s[sel])
    return np.abs(grid[..., sel] - gref).max() / np.abs(gref).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_series_against_exact_sum_and_oracle(torch_cuda, precision):
    from paper_1404_7357_gb300 import cfft
    if precision == "fp64":
        wl = workloads.strip_fp64(n=1024, n_rho=256, rho_max=10.0)
    else:
        wl = cc.small_patch("fp32", n=1024, n_rho=256, rho_max=4.0, q_max=3)
    ref, _, _ = cc.oracle_table(wl)
    res = {}
    for mode in (1, 2):
        # Lagrange back-projection: the grid then holds g(s_k) itself (no precorrection)
        ctx, got = cc.gpu_table(wl, options={cfft.OPT_CONTOUR_SERIES: mode, cfft.OPT_BP_KERNEL: 1})
        info = ctx.info()
        assert info["contour_series"] == mode - 1
        ffts = info["taylor_order"] + (2 if mode == 2 else 1)
        res[mode] = (_grid_error(ctx, wl), cc.rel_err_per_pair(got, ref).max(), ffts)
    print(precision, "Taylor (grid, table, FFTs) =", res[1], "Chebyshev =", res[2])
    grid_tol = 1e-11 if precision == "fp64" else 2e-5
    for mode in (1, 2):
        assert res[mode][0] < grid_tol and res[mode][1] < TOL[precision]
    assert res[2][2] < res[1][2]          # fewer transforms for the same bound


def test_automatic_choice_and_explicit_order(torch_cuda):
    wl = workloads.strip_fp64(n=1024, n_rho=256, rho_max=10.0)
    ctx, _ = cc.gpu_table(wl)
    auto = ctx.info()
    assert auto["contour_series"] == 1    # height * rho_max = 2.7: 16 Chebyshev FFTs against 25
    wl.extras["taylor"] = 6
    ctx, _ = cc.gpu_table(wl)
    fixed = ctx.info()
    assert fixed["contour_series"] == 0 and fixed["taylor_order"] == 6


def test_chebyshev_error_falls_with_degree(torch_cuda):
    from paper_1404_7357_gb300 import cfft
    wl = workloads.strip_fp64(n=1024, n_rho=128, rho_max=10.0)
    errs = []
    for deg in (0, 1, 2, 4, 8, 12):
        wl.extras["taylor"] = deg
        ctx, _ = cc.gpu_table(wl, options={cfft.OPT_CONTOUR_SERIES: 2})
        assert ctx.info()["contour_series"] == 1
        errs.append(_grid_error(ctx, wl))
    print("Chebyshev degree 0, 1, 2, 4, 8, 12: grid error", errs)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    # remainder bound at degree 12, a = height rho_max / 2 = 1.37: 2 e^a I_13(a) = 8e-12
    assert errs[-1] < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sub_fft_length_option(torch_cuda, precision):
    """Eq. 23's split of the length-P transform into P / L residue classes of its outputs
    gives the same grid for every sub-FFT length L (cfft_set_option FFT_SUB_LEN); lengths
    that are not powers of two, too short or too long, or not dividing P are refused."""
    from paper_1404_7357_gb300 import cfft
    if precision == "fp64":
        wl = workloads.strip_fp64(n=1024, n_rho=256, rho_max=10.0)
    else:
        wl = cc.small_patch("fp32", n=1024, n_rho=256, rho_max=4.0, q_max=3)
    ref, _, _ = cc.oracle_table(wl)
    grid_tol = 1e-11 if precision == "fp64" else 2e-5
    for sub_len in (64, 512, 4096):
        ctx, got = cc.gpu_table(wl, options={cfft.OPT_FFT_SUB_LEN: sub_len, cfft.OPT_BP_KERNEL: 1})
        assert ctx.info()["sub_len"] == sub_len
        ge, te = _grid_error(ctx, wl), cc.rel_err_per_pair(got, ref).max()
        print(precision, "L =", sub_len, "grid", ge, "table", te)
        assert ge < grid_tol and te < TOL[precision]
    prec = cfft.CFFT_FP64 if precision == "fp64" else cfft.CFFT_FP32_MIXED
    for bad in (96, 32, 32768, 65536):
        ctx = cc.gpu_context(wl, options={cfft.OPT_FFT_SUB_LEN: bad})
        with pytest.raises(cfft.CfftError) as ei:
            ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, prec, 1)
        assert ei.value.status == 1
