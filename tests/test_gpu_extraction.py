"""Z^l on the GPU (Sections II and III-A): tables tabulated with the effective homogeneous
medium and its image through the ground plane extracted from the slab's Green's function
(cfft_set_green_extraction), through the C ABI:

- the strip (FP64) and the 4-MBF patch (FP32) against the oracle's tables computed with
  the same remainder Green's function;
- an air slab (eps_r = 1): the remainder is zero, so is the table;
- the point of the split: with the charge term removed, the remainder's table is
  insensitive to the truncation beta_max where the full table is not;
- the substrate derivatives of the remainder against finite differences of its table;
- the Cartesian tabulation honours the same extraction.
"""
import dataclasses

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


def _extracted_table(wl, options=None):
    from paper_1404_7357_gb300 import cfft
    ctx = cc.gpu_context(wl, options=options)
    ctx.set_green_extraction(True)
    prec = cfft.CFFT_FP64 if wl.precision == "fp64" else cfft.CFFT_FP32_MIXED
    ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, prec, wl.rotation_classes)
    return ctx, ctx.copy_table(host=True).numpy()


def _oracle_remainder_table(wl):
    from oracle import contour as oc
    from oracle import green as og
    from oracle import reaction as orx
    c, s = wl.contour, wl.substrate
    nodes = oc.contour_nodes(c.n, c.beta_max, c.beta_p, c.height)
    hq = orx.harmonics(cc.oracle_basis(wl.element), nodes["beta_c"], wl.qs, cc.oracle_n_alpha(wl), s.eps_r, s.h,
                       s.k0, green_fn=og.layered_remainder(), workers=cc.oracle_workers())
    z = orx.table_bessel(hq, wl.qs, nodes["beta_c"], nodes["weight"], wl.rho)
    m = z.shape[0]
    return z.reshape(1, m * m, len(wl.qs), len(wl.rho))


@pytest.mark.parametrize("case", ["strip-fp64", "patch-fp32"])
def test_remainder_table_against_oracle(torch_cuda, case):
    if case == "strip-fp64":
        wl = workloads.strip_fp64(n=1024, n_rho=256, rho_max=4.0, q_max=3)
    else:
        wl = cc.small_patch("fp32", n=1024, n_rho=256, rho_max=4.0, q_max=2)
    _, got = _extracted_table(wl)
    ref = _oracle_remainder_table(wl)
    err = cc.rel_err_per_pair(got, ref).max()
    print(case, "Z^l table vs oracle: %.3g" % err)
    assert err < TOL[wl.precision]


def test_air_slab_remainder_vanishes(torch_cuda):
    base = workloads.strip_fp64(n=1024, n_rho=128, rho_max=3.0, q_max=2)
    sub = workloads.Substrate(eps_r=1.0, h=0.05)
    wl = dataclasses.replace(base, substrate=sub, contour=workloads.default_contour(sub, 1024, beta_p_factor=1.6))
    full = cc.gpu_table(wl)[1]
    _, rem = _extracted_table(wl)
    ratio = np.abs(rem).max() / np.abs(full).max()
    print("air slab: max |Z^l| / max |Z| = %.3g" % ratio)
    assert ratio < 1e-11


def test_remainder_is_insensitive_to_the_truncation(torch_cuda):
    """Strip on eps_r 2.2: tables truncated at beta_max = 4 k_d and 10 k_d (the same node
    spacing and contour), full slab vs remainder: the remainder moves far less."""
    base = workloads.strip_fp64(n=1024, n_rho=256, rho_max=2.0, q_max=2)
    s = base.substrate
    step = 5.0 * s.k_d / 1024
    moves = {}
    for extract in (False, True):
        tabs = []
        for factor in (4.0, 10.0):
            n = int(round(factor * s.k_d / step / 32.0)) * 32
            c = dataclasses.replace(base.contour, n=n, beta_max=n * step)
            wl = dataclasses.replace(base, contour=c)
            tabs.append(_extracted_table(wl)[1] if extract else cc.gpu_table(wl)[1])
        moves[extract] = np.abs(tabs[0] - tabs[1]).max() / np.abs(tabs[1]).max()
    print("change from beta_max 4 k_d to 10 k_d: full %.3g, remainder %.3g" % (moves[False], moves[True]))
    assert moves[True] < 0.2 * moves[False]


def test_remainder_derivatives_against_finite_differences(torch_cuda):
    from paper_1404_7357_gb300 import cfft
    wl = workloads.strip_fp64(n=1024, n_rho=128, rho_max=3.0, q_max=2)
    ctx, _ = _extracted_table(wl, options={cfft.OPT_DERIVATIVES: 1})
    d_eps = ctx.derivative_table(1).cpu().numpy()
    d_h = ctx.derivative_table(2).cpu().numpy()
    s = wl.substrate
    for which, step, got in (("eps_r", 1e-5, d_eps), ("h", 1e-7, d_h)):
        vals = []
        for sign in (1, -1):
            sub = dataclasses.replace(s, eps_r=s.eps_r + sign * step) if which == "eps_r" else \
                dataclasses.replace(s, h=s.h + sign * step)
            vals.append(_extracted_table(dataclasses.replace(wl, substrate=sub))[1])
        fd = (vals[0] - vals[1]) / (2 * step)
        err = np.abs(got - fd).max() / np.abs(fd).max()
        print("d Z^l / d %s vs central difference: %.3g" % (which, err))
        assert err < 1e-5


def test_cartesian_tabulation_honours_the_extraction(torch_cuda):
    from oracle import cartesian as oca
    from oracle import green as og
    from paper_1404_7357_gb300 import cfft
    wl = workloads.strip_fp64(n=1024)
    ctx = cc.gpu_context(wl)
    ctx.set_green_extraction(True)
    ctx.tabulate_cartesian(64, 2.0, cfft.CFFT_FP64, taylor_order=10)
    got = ctx.cartesian_table().cpu().numpy()
    c, s = wl.contour, wl.substrate
    ref, _ = oca.table(cc.oracle_basis(wl.element), s.eps_r, s.h, s.k0, c.beta_max, c.beta_p, c.height, 64, 10,
                       green_fn=og.layered_remainder())
    err = np.abs(got - ref.reshape(got.shape)).max() / np.abs(ref).max()
    print("Cartesian Z^l vs oracle: %.3g" % err)
    assert err < 1e-10
