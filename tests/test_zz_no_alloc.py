"""cfft_backproject_static: the back-projection for callers that cannot allocate.

A caller that lives inside an application that owns every device allocation,
or runs a real-time loop, cannot let the library call cudaMalloc.  This entry point keeps its scratch in a fixed
device array inside the library; the caller brings the transform grid and
the output table.  Its result must match the table that cfft_tabulate_reactions
produced from the same grid, on two calls in a row (the second call reuses
the array the first one left behind).  This file is collected last.
"""
import math

import numpy as np
import pytest

from tests import cfft_cases as cc

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_static_backprojection_matches_tabulation(torch_cuda, precision):
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch(precision, n=1024, n_rho=256, rho_max=4.0, q_max=3)
    # the static entry interpolates with Lagrange stencils: the tabulation it is compared
    # with uses them too (its grid then holds g(s_k) itself)
    ctx, ref = cc.gpu_table(wl, options={cfft.OPT_BP_KERNEL: 1})   # the existing entry point's table
    info = ctx.info()
    grid = ctx.debug_buffer("grid").contiguous()  # (classes, pairs, harmonics, 2K+1), device
    c = wl.contour
    beta_abs = math.hypot(c.beta_max, c.height)
    series_per_q = grid.shape[0] * grid.shape[1]
    out = torch.empty(grid.shape[:3] + (wl.n_rho,), dtype=grid.dtype, device=grid.device)
    for call in range(2):
        out.fill_(complex(float("nan"), float("nan")))
        cfft.backproject_static(grid, out, series_per_q, wl.q_max, wl.rho_max, info["grid_half"],
                                info["delta_s"], info["sigma"], info["bp_taps"], beta_abs)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all(), "call %d left entries unwritten" % call
        err = cc.rel_err_per_pair(got, ref).max()
        print(precision, "call", call, "static vs tabulate rel err", err)
        assert err < TOL[precision]


def test_static_backprojection_rejects_oversized_requests(torch_cuda):
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    grid = torch.zeros((1, 1, 1, 101), dtype=torch.complex64, device="cuda:0")
    table = torch.zeros((1, 1, 1, 64), dtype=torch.complex64, device="cuda:0")
    # far more angular nodes than the fixed scratch holds: rejected before any work is queued
    wide = torch.zeros((1, 1, 1, 2 * 200000 + 1), dtype=torch.complex64, device="cuda:0")
    with pytest.raises(cfft.CfftError) as ei:
        cfft.backproject_static(wide, table, 1, 0, 1.0e5, 200000, 1.0, 4, 8, 100.0)
    assert ei.value.status == 1
    # a grid that does not hold [series][2*grid_half+1]: refused by the binding
    with pytest.raises(ValueError):
        cfft.backproject_static(grid, table, 1, 0, 1.0e5, 200000, 1.0, 4, 8, 100.0)
    # rho_max beyond the grid half-width: rejected as well
    with pytest.raises(cfft.CfftError) as ei:
        cfft.backproject_static(grid, table, 1, 0, 10.0, 50, 0.1, 4, 8, 10.0)
    assert ei.value.status == 1
