"""Failure detection on the GPU without a fault: a device-side wait that nothing ends
runs out after its bound and the library reports CFFT_ERR_TIMEOUT; out-of-memory
injected on the host makes the call in progress return CFFT_ERR_OOM.  Either way the
context stays usable.  Nothing here traps, faults or waits without a bound."""
import numpy as np
import pytest

import workloads
from tests import cfft_cases as cc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_bounded_wait_runs_out_and_context_survives(torch_cuda):
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch("fp32", n=1024, n_rho=128, rho_max=3.0, q_max=2)
    ctx = cc.gpu_context(wl)
    for polls in (1, 4096):
        with pytest.raises(cfft.CfftError) as ei:
            ctx.selftest_bounded_wait(polls)
        assert ei.value.status == 6                     # CFFT_ERR_TIMEOUT
    with pytest.raises(cfft.CfftError) as ei:
        ctx.selftest_bounded_wait(0)                    # a bound of zero tries is refused
    assert ei.value.status == 1
    # the same context tabulates correctly afterwards
    ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP32_MIXED, 1)
    got = ctx.copy_table(host=True).numpy()
    ref, _, _ = cc.oracle_table(wl)
    err = cc.rel_err_per_pair(got, ref).max()
    print("after the timeout: table rel err", err)
    assert err < 1e-5


def test_injected_allocation_failures_leave_contexts_usable(torch_cuda):
    """Out-of-memory injected on the host (no allocation attempted) at several points of a
    first tabulation, and at the fill's scratch: each call returns CFFT_ERR_OOM, and the
    same context then tabulates and fills as an untouched one does."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch("fp32", n=1024, n_rho=256, rho_max=3.0, q_max=2, rotation_classes=4)
    ref_ctx, ref = cc.gpu_table(wl)
    pos = torch.tensor(workloads.poisson_disc(20, 1.4, 0.4, seed=7), device="cuda:0")
    rot = torch.tensor(workloads.rotations(20, seed=7), device="cuda:0")
    n = 20 * wl.element.n_mbf
    zref = torch.empty((n, n), dtype=torch.complex64, device="cuda:0")
    ref_ctx.fill_reduced_matrix(pos, rot, zref)
    try:
        for after in (0, 3, 9):
            ctx = cc.gpu_context(wl)
            cfft.test_fail_allocation(after)
            with pytest.raises(cfft.CfftError) as ei:
                ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP32_MIXED, 4)
            assert ei.value.status == 3                      # CFFT_ERR_OOM
            cfft.test_fail_allocation(-1)
            ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP32_MIXED, 4)
            got = ctx.copy_table(host=True).numpy()
            assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()
            cfft.test_fail_allocation(0)                     # the fill's scratch, first fill
            z = torch.empty_like(zref)
            with pytest.raises(cfft.CfftError) as ei:
                ctx.fill_reduced_matrix(pos, rot, z)
            assert ei.value.status == 3
            ctx.fill_reduced_matrix(pos, rot, z)
            assert ((z - zref).abs().max() <= 1e-6 * zref.abs().max()).item()
            print("allocation failure after", after, "allocations: OOM reported, context usable")
    finally:
        cfft.test_fail_allocation(-1)
