"""The paper's own 2-D Cartesian C-FFT on the GPU (Section III-B-2/3, Eq. 21-24,
Appendix I), through the C ABI:

- the whole table against the oracle's (same grid, Taylor order and contour): the strip in
  FP64 and the 4-MBF patch (16 pairs) in FP32, every lattice point;
- the second-order interpolation fill against the oracle's interpolation of its own table;
- the Cartesian tabulation against the harmonic one on the same contour: both evaluate
  the contour integral of Eq. 9, so on a fine Cartesian grid their reduced matrices agree
  to the Cartesian rectangle rule's error (first to second order in dk on the circles
  |k| = beta_p and beta_max);
- refusals: a rho_max outside the table, and a fill pair beyond rho_max.
"""
import math

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


def _oracle_table(wl, n_grid, order):
    from oracle import cartesian as oca
    c, s = wl.contour, wl.substrate
    return oca.table(cc.oracle_basis(wl.element), s.eps_r, s.h, s.k0, c.beta_max, c.beta_p, c.height,
                     n_grid, order)


@pytest.mark.parametrize("case", ["strip-fp64", "patch-fp32"])
def test_cartesian_table_against_oracle(torch_cuda, case):
    from paper_1404_7357_gb300 import cfft
    if case == "strip-fp64":
        wl = workloads.strip_fp64(n=1024)
        prec, n_grid, order, rho = cfft.CFFT_FP64, 64, 10, 2.0
    else:
        wl = cc.small_patch("fp32", n=1024)
        prec, n_grid, order, rho = cfft.CFFT_FP32_MIXED, 64, 6, 1.4
    precision = "fp64" if prec == cfft.CFFT_FP64 else "fp32"
    ctx = cc.gpu_context(wl)
    info = ctx.tabulate_cartesian(n_grid, rho, prec, taylor_order=order)
    assert info["n_table"] == 2 * n_grid and info["monomials"] == (order + 1) * (order + 2) // 2
    got = ctx.cartesian_table().cpu().numpy().astype(np.complex128)
    ref, x = _oracle_table(wl, n_grid, order)
    m = wl.element.n_mbf
    ref = ref.reshape(m * m, 2 * n_grid, 2 * n_grid)
    assert abs(info["x0"] - x[0]) < 1e-12 and abs(info["step"] - (x[1] - x[0])) < 1e-12
    err = (np.abs(got - ref).reshape(m * m, -1).max(-1) / np.abs(ref).reshape(m * m, -1).max(-1)).max()
    print(case, "Cartesian table vs oracle: rel err %.3g" % err, info)
    assert err < TOL[precision]


def test_cartesian_fill_against_oracle(torch_cuda):
    torch = torch_cuda
    from oracle import cartesian as oca
    from paper_1404_7357_gb300 import cfft
    wl = workloads.strip_fp64(n=1024)
    n_grid, order, rho = 64, 10, 2.0
    ctx = cc.gpu_context(wl)
    ctx.tabulate_cartesian(n_grid, rho, cfft.CFFT_FP64, taylor_order=order)
    pos = np.array([[0.0, 0.0], [0.71, 0.33], [-0.52, 1.04], [0.6, -0.4]])     # pairs within 2
    a = len(pos)
    z = torch.zeros((a, a), dtype=torch.complex128, device="cuda:0")
    ctx.fill_cartesian(torch.tensor(pos, device="cuda:0"), z)
    tab, x = _oracle_table(wl, n_grid, order)
    ref = np.zeros((a, a), dtype=np.complex128)
    for i in range(a):
        for j in range(a):
            d = pos[i] - pos[j]
            ref[i, j] = oca.interpolate(tab, x, np.array([d[0]]), np.array([d[1]]))[0, 0, 0]
    err = np.abs(z.cpu().numpy() - ref).max() / np.abs(ref).max()
    print("Cartesian fill vs oracle interpolation: %.3g" % err)
    assert err < 1e-11
    with pytest.raises(cfft.CfftError) as ei:       # a pair beyond rho_max
        far = np.array([[0.0, 0.0], [2.5, 0.0]])
        ctx.fill_cartesian(torch.tensor(far, device="cuda:0"),
                           torch.zeros((2, 2), dtype=torch.complex128, device="cuda:0"))
    assert ei.value.status == 1
    with pytest.raises(cfft.CfftError):               # rho_max outside a 64-point table
        ctx.tabulate_cartesian(n_grid, 5.0, cfft.CFFT_FP64, taylor_order=order)


def test_cartesian_agrees_with_the_harmonic_tabulation(torch_cuda):
    """Strip element, one contour for both (height 6 Cartesian steps): the harmonic table
    (|q| <= 40, fine contour) filled at a few relative positions against the Cartesian
    table at the same positions, on two Cartesian grids."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    base = workloads.strip_fp64()
    c = base.contour
    import dataclasses
    height = 6 * 2 * c.beta_max / 512
    wl = dataclasses.replace(base, contour=dataclasses.replace(c, n=8192, height=height), q_max=40, n_rho=1024,
                             rho_max=3.0)
    ctx = cc.gpu_context(wl, options={cfft.OPT_N_ALPHA: 256})
    ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP64, 1)
    step = math.pi / (2 * c.beta_max)
    pts = [(2 * step * i, 2 * step * j) for i in (0, 4, 16, 30) for j in (0, 2, 10)]
    pos = np.array([[0.0, 0.0]] + [list(p) for p in pts])
    a = len(pos)
    zh = torch.zeros((a, a), dtype=torch.complex128, device="cuda:0")
    ctx.fill_reduced_matrix(torch.tensor(pos, device="cuda:0"), None, zh)
    harm = zh.cpu().numpy()[1:, 0]
    errs = []
    for n_grid in (256, 512):
        ctx.tabulate_cartesian(n_grid, 2.5, cfft.CFFT_FP64, taylor_order=16)
        zc = torch.zeros((a, a), dtype=torch.complex128, device="cuda:0")
        ctx.fill_cartesian(torch.tensor(pos, device="cuda:0"), zc)
        cart = zc.cpu().numpy()[1:, 0]
        errs.append(np.abs(cart - harm).max() / np.abs(harm).max())
    print("Cartesian vs harmonic tabulation: n 256 %.3g, n 512 %.3g" % tuple(errs))
    assert errs[1] < 1e-3 and errs[0] / errs[1] > 2.5
