"""Batched sweep (cfft_tabulate_batch): many substrates and frequencies with uneven
contour lengths in multi-item / persistent launches, replayed from a CUDA graph.

Each item's table must agree with the single-item tabulation of the same item
(itself oracle-checked) within the precision tolerance, a replay with new
substrate values must track them, autotuning must not change the result, and
one item is compared with the FP64 oracle directly.
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


def _items(n_items=5, seed=9):
    its = workloads.sweep_items(n_freq=n_items, n_sub=1, seed=seed, rho_max=3.0, n_base=256,
                                n_levels=3)
    rng = np.random.default_rng(seed)
    for it in its:  # spread the substrates too
        it["eps_r"] = float(rng.uniform(2.0, 10.0))
        kd = it["k0"] * np.sqrt(it["eps_r"])
        it["beta_max"] = 5.0 * kd
        step = it["beta_max"] / it["n"]
        it["beta_p"] = round(1.3 * kd / step) * step
        it["height"] = 6.0 * step
    return its


def _single(cfft, el, it, q_max, rho_max, n_rho, prec, n_alpha):
    ctx = cfft.Context(0)
    ctx.set_substrate(it["eps_r"], it["h"], it["k0"])
    ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
    ctx.build_contour(it["n"], it["beta_max"], it["beta_p"], it["height"], int(it.get("taylor_order", -1)))
    ctx.set_option(cfft.OPT_N_ALPHA, n_alpha)
    ctx.tabulate_reactions(q_max, rho_max, n_rho, prec, 1)
    return ctx.copy_table(host=True).numpy()[0]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_matches_single_tabulations(torch_cuda, precision):
    from paper_1404_7357_gb300 import cfft
    prec = cfft.CFFT_FP64 if precision == "fp64" else cfft.CFFT_FP32_MIXED
    el = workloads.patch_rooftops()
    items = _items()
    q_max, rho_max, n_rho = 3, 3.0, 256
    ctx = cfft.Context(0)
    ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
    ctx.set_option(cfft.OPT_N_ALPHA, 128)
    out = ctx.tabulate_batch(items, q_max, rho_max, n_rho, prec, graph=False)
    got = out.cpu().numpy()
    print(precision, "batch info", ctx.batch_info(), [it["n"] for it in items])
    for i, it in enumerate(items):
        ref = _single(cfft, el, it, q_max, rho_max, n_rho, prec, 128)
        err = np.abs(got[i].astype(np.complex128) - ref).max() / np.abs(ref).max()
        print(precision, "item", i, "n", it["n"], "eps", round(it["eps_r"], 3), "rel err", err)
        assert err < TOL[precision]


def test_batch_graph_replay_tracks_new_parameters(torch_cuda):
    from paper_1404_7357_gb300 import cfft
    el = workloads.patch_rooftops()
    items = _items(4, seed=11)
    q_max, rho_max, n_rho = 2, 3.0, 128
    ctx = cfft.Context(0)
    ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
    ctx.set_option(cfft.OPT_N_ALPHA, 128)
    out = ctx.tabulate_batch(items, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, graph=True)
    first = out.cpu().numpy().copy()
    # same structure, new substrates: the captured graph is replayed on refreshed parameters
    for it in items:
        it["h"] *= 1.1
    out = ctx.tabulate_batch(items, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, out=out, graph=True)
    second = out.cpu().numpy()
    assert np.abs(second - first).max() > 1e-3 * np.abs(first).max()
    for i, it in enumerate(items):
        ref = _single(cfft, el, it, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, 128)
        err = np.abs(second[i].astype(np.complex128) - ref).max() / np.abs(ref).max()
        assert err < TOL["fp32"]
    # and an autotuned plan gives the same tables
    out2 = ctx.tabulate_batch(items, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, graph=True,
                              autotune=True)
    info = ctx.batch_info()
    print("autotuned", info)
    tuned = out2.cpu().numpy()
    assert np.abs(tuned - second).max() < TOL["fp32"] * np.abs(second).max()


def test_batch_per_item_angle_counts(torch_cuda):
    """Automatic angle counts: the sweep runs the tensor-core integrand at 128 angles for
    the items whose spectra need no more and at 256 for the others (one launch each); every
    item against the single tabulation of that item, which chooses its own count."""
    from paper_1404_7357_gb300 import cfft
    el = workloads.patch_rooftops()
    items = _items(6, seed=21)
    items[0]["eps_r"], items[-1]["eps_r"] = 2.0, 10.0       # both ends of the substrate range
    for it in (items[0], items[-1]):
        kd = it["k0"] * np.sqrt(it["eps_r"])
        it["beta_max"] = 5.0 * kd
        step = it["beta_max"] / it["n"]
        it["beta_p"] = round(1.3 * kd / step) * step
        it["height"] = 6.0 * step
    q_max, rho_max, n_rho = 16, 3.0, 256
    ctx = cfft.Context(0)
    ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
    got = ctx.tabulate_batch(items, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, graph=True).cpu().numpy()
    counts = []
    for i, it in enumerate(items):
        c1 = cfft.Context(0)
        c1.set_substrate(it["eps_r"], it["h"], it["k0"])
        c1.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
        c1.build_contour(it["n"], it["beta_max"], it["beta_p"], it["height"], -1)
        c1.tabulate_reactions(q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, 1)
        ref = c1.copy_table(host=True).numpy()[0].astype(np.complex128)
        counts.append(c1.info()["n_alpha"])
        err = np.abs(got[i].astype(np.complex128) - ref).max() / np.abs(ref).max()
        print("item", i, "eps", round(it["eps_r"], 2), "n_alpha", counts[-1], "rel err %.3g" % err)
        assert err < 2e-6
    assert 128 in counts and 256 in counts


def test_batch_item_against_oracle(torch_cuda):
    from paper_1404_7357_gb300 import cfft
    el = workloads.patch_rooftops()
    it = _items(1, seed=13)[0]
    q_max, rho_max, n_rho = 2, 2.5, 96
    ctx = cfft.Context(0)
    ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
    got = ctx.tabulate_batch([it], q_max, rho_max, n_rho, cfft.CFFT_FP64, graph=True).cpu().numpy()[0]
    wl = workloads.TableWorkload("batch-item", workloads.Substrate(it["eps_r"], it["h"], it["k0"]), el,
                                 workloads.ContourSpec(it["n"], it["beta_max"], it["beta_p"], it["height"]),
                                 q_max, rho_max, n_rho, "fp64")
    ref, _, _ = cc.oracle_table(wl)
    err = cc.rel_err_per_pair(got[None], ref).max()
    print("batch item vs oracle", err)
    assert err < TOL["fp64"]


def test_batch_backprojection_forms(torch_cuda):
    """FP32-mixed batch with the back-projection's products on the tensor cores and on
    the FP32 pipe (CFFT_OPT_BP_SIMT): both against single tabulations, several row tiles."""
    from paper_1404_7357_gb300 import cfft
    el = workloads.patch_rooftops()
    items = _items(3, seed=13)
    q_max, rho_max, n_rho = 2, 4.0, 600
    refs = [_single(cfft, el, it, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, 128) for it in items]
    for simt in (0, 1):
        ctx = cfft.Context(0)
        ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
        ctx.set_option(cfft.OPT_N_ALPHA, 128)
        ctx.set_option(cfft.OPT_BP_SIMT, simt)
        got = ctx.tabulate_batch(items, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, graph=True).cpu().numpy()
        assert ctx.batch_info()["bp_tc"] == 1 - simt
        for i in range(len(items)):
            err = np.abs(got[i].astype(np.complex128) - refs[i]).max() / np.abs(refs[i]).max()
            print("bp simt", simt, "item", i, "rel err vs single", err)
            assert err < 2e-6
