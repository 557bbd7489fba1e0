"""Failure detection on the GPU without a fault: a device-side wait that nothing ends
runs out after its bound and the library reports CFFT_ERR_TIMEOUT; the context stays
usable (a tabulation right after matches the oracle).  Nothing here traps, faults or
waits without a bound."""
import numpy as np
import pytest

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
