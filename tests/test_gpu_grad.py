"""Gradients of an array objective through the differentiable fill (GPU).

L = sum_i |(Z' v - t)_i|^2 for seeded complex-normal v, t.  The analytic
gradient of ReducedMatrix (hand-written adjoint of the fill plus forward-mode
substrate derivative tables) is checked against central finite differences of
the GPU forward pass and against finite differences of the FP64 oracle's exact
fill (contour held fixed in every evaluation).
"""
import math

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


def _setup(precision, torch, n_el=8, radius=1.3):
    from paper_1404_7357_gb300.autograd import FillProblem
    wl = cc.small_patch(precision, n=512, n_rho=256, rho_max=2.7, q_max=3, rotation_classes=4)
    pos = workloads.poisson_disc(n_el, radius, 0.5, seed=51)
    rot = workloads.rotations(n_el, seed=51)
    prob = FillProblem(wl.element, wl.substrate.k0, wl.contour, wl.q_max, wl.rho_max, wl.n_rho,
                       precision, rot=torch.tensor(rot, device="cuda:0"))
    m = wl.element.n_mbf
    v = torch.tensor(workloads.complex_normal(n_el * m, 52), device="cuda:0")
    t = torch.tensor(workloads.complex_normal(n_el * m, 53), device="cuda:0")
    return wl, pos, rot, prob, v, t


def _loss(torch, prob, pos_t, eh_t, v, t):
    from paper_1404_7357_gb300.autograd import ReducedMatrix
    z = ReducedMatrix.apply(pos_t, eh_t, prob)
    r = z.to(torch.complex128) @ v - t
    return (r.abs() ** 2).sum()


def test_gradient_matches_finite_differences_fp64(torch_cuda):
    torch = torch_cuda
    wl, pos, rot, prob, v, t = _setup("fp64", torch)
    s = wl.substrate
    pos_t = torch.tensor(pos, device="cuda:0", requires_grad=True)
    eh_t = torch.tensor([s.eps_r, s.h], dtype=torch.float64, device="cuda:0", requires_grad=True)
    loss = _loss(torch, prob, pos_t, eh_t, v, t)
    loss.backward()
    gpos = pos_t.grad.cpu().numpy()
    geh = eh_t.grad.cpu().numpy()

    def f(p, eh):
        with torch.no_grad():
            return float(_loss(torch, prob, torch.tensor(p, device="cuda:0"),
                               torch.tensor(eh, dtype=torch.float64, device="cuda:0"), v, t))

    eh0 = np.array([s.eps_r, s.h])
    for (i, k) in [(0, 0), (3, 1), (5, 0), (7, 1)]:
        d = 1e-6
        pp, pm = pos.copy(), pos.copy()
        pp[i, k] += d
        pm[i, k] -= d
        fd = (f(pp, eh0) - f(pm, eh0)) / (2 * d)
        assert abs(fd - gpos[i, k]) < 1e-6 * max(1.0, abs(fd)) + 1e-7 * np.abs(gpos).max(), (i, k, fd, gpos[i, k])
    for j, d in [(0, 1e-6), (1, 1e-7)]:
        ep, em = eh0.copy(), eh0.copy()
        ep[j] += d
        em[j] -= d
        fd = (f(pos, ep) - f(pos, em)) / (2 * d)
        print("substrate grad", j, fd, geh[j])
        assert abs(fd - geh[j]) < 1e-6 * abs(fd), (j, fd, geh[j])
    # translation invariance: the position gradient sums to zero
    assert np.abs(gpos.sum(0)).max() < 1e-9 * np.abs(gpos).max()


def test_gradient_matches_oracle_finite_differences(torch_cuda):
    torch = torch_cuda
    wl, pos, rot, prob, v, t = _setup("fp64", torch, n_el=5, radius=1.1)
    s = wl.substrate
    pos_t = torch.tensor(pos, device="cuda:0", requires_grad=True)
    eh_t = torch.tensor([s.eps_r, s.h], dtype=torch.float64, device="cuda:0", requires_grad=True)
    _loss(torch, prob, pos_t, eh_t, v, t).backward()
    gpos = pos_t.grad.cpu().numpy()
    geh = eh_t.grad.cpu().numpy()
    vn, tn = v.cpu().numpy(), t.cpu().numpy()

    import copy
    from oracle import fill as ofill

    def oracle_loss(p, eps_r, h):
        w2 = copy.deepcopy(wl)
        w2.substrate = workloads.Substrate(eps_r=eps_r, h=h, k0=s.k0)  # contour unchanged
        nodes, hq = cc.oracle_harmonics(w2, classes=(0, 1, 2, 3))
        z = ofill.full_matrix(hq, w2.qs, nodes["beta_c"], nodes["weight"], p, rot)
        r = z @ vn - tn
        return float(np.sum(np.abs(r) ** 2))

    for j, d in [(0, 1e-5), (1, 1e-6)]:
        ep = [s.eps_r, s.h]
        em = [s.eps_r, s.h]
        ep[j] += d
        em[j] -= d
        fd = (oracle_loss(pos, *ep) - oracle_loss(pos, *em)) / (2 * d)
        print("oracle substrate fd", j, fd, geh[j])
        assert abs(fd - geh[j]) < 1e-5 * abs(fd)
    i, k, d = 2, 1, 1e-6
    pp, pm = pos.copy(), pos.copy()
    pp[i, k] += d
    pm[i, k] -= d
    fd = (oracle_loss(pp, s.eps_r, s.h) - oracle_loss(pm, s.eps_r, s.h)) / (2 * d)
    print("oracle position fd", fd, gpos[i, k])
    assert abs(fd - gpos[i, k]) < 1e-5 * max(abs(fd), 1e-3 * np.abs(gpos).max())


def test_fp32_gradient_close_to_fp64(torch_cuda):
    torch = torch_cuda
    grads = {}
    for prec in ("fp64", "fp32"):
        wl, pos, rot, prob, v, t = _setup(prec, torch)
        s = wl.substrate
        pos_t = torch.tensor(pos, device="cuda:0", requires_grad=True)
        eh_t = torch.tensor([s.eps_r, s.h], dtype=torch.float64, device="cuda:0", requires_grad=True)
        _loss(torch, prob, pos_t, eh_t, v, t).backward()
        grads[prec] = (pos_t.grad.cpu().numpy(), eh_t.grad.cpu().numpy())
    ep, eh = grads["fp64"]
    fp, fh = grads["fp32"]
    # float32 tables (~5e-7) differentiated through the interpolation slope: ~2e-4 of max
    print("fp32 vs fp64 gradient", np.abs(fp - ep).max() / np.abs(ep).max(), np.abs(fh - eh) / np.abs(eh))
    assert np.abs(fp - ep).max() < 1e-3 * np.abs(ep).max()
    assert np.all(np.abs(fh - eh) < 1e-3 * np.abs(eh))


def _adjoint(torch, ctx, pos, rot, g, block):
    from paper_1404_7357_gb300 import cfft
    ctx.set_option(cfft.OPT_FILL_BLOCK, block)
    rt = None if rot is None else torch.tensor(rot, device="cuda:0")
    gp, gt = ctx.fill_backward(torch.tensor(pos, device="cuda:0"), rt, g)
    return gp.cpu().numpy(), gt.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_bucketed_adjoint_matches_per_row(torch_cuda, precision):
    """The adjoint over the fill's buckets against the per-row adjoint: row blocks that
    split the elements raggedly, a gradient with a padded odd leading dimension (no
    vector loads), four rotation classes and the substrate channels."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch(precision, n=1024, n_rho=1024, rho_max=9.0, q_max=4, rotation_classes=4)
    ctx = cc.gpu_context(wl, options={cfft.OPT_DERIVATIVES: 1})
    prec = cfft.CFFT_FP64 if precision == "fp64" else cfft.CFFT_FP32_MIXED
    ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, prec, 4)
    pos = workloads.poisson_disc(300, 4.4, 0.3, seed=41)
    rot = workloads.rotations(len(pos), seed=41)
    a, m = len(pos), 4
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    gfull = torch.tensor(workloads.complex_normal(a * m * (a * m + 1), 42).reshape(a * m, a * m + 1),
                         device="cuda:0").to(dt)
    ref_p, ref_t = _adjoint(torch, ctx, pos, rot, gfull[:, :a * m].contiguous(), -1)
    # FP32: both sides form each pair's term in float32 and sum ~10^6 of them with
    # cancellation (the substrate terms carry the diagonal too), in different orders
    tol_p, tol_t = (1e-11, 1e-11) if precision == "fp64" else (2e-5, 5e-5)
    for block, g in ((0, gfull[:, :a * m].contiguous()), (37, gfull[:, :a * m]), (1000, gfull[:, :a * m])):
        gp, gt = _adjoint(torch, ctx, pos, rot, g, block)
        ep = np.abs(gp - ref_p).max() / np.abs(ref_p).max()
        et = np.abs(gt - ref_t) / np.abs(ref_t)
        print(precision, "block", block, "ld", g.stride(0), "pos", ep, "eps/h", et)
        assert ep < tol_p and np.all(et < tol_t)
    assert np.abs(ref_p.sum(0)).max() < 1e-6 * np.abs(ref_p).max()


@pytest.mark.parametrize("m,taps", [(1, 8), (2, 12), (2, 16)])
def test_bucketed_adjoint_m_and_taps(torch_cuda, m, taps):
    import dataclasses
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch("fp64", n=1024, n_rho=512, rho_max=5.0, q_max=3, rotation_classes=4)
    el = wl.element
    wl = dataclasses.replace(wl, element=dataclasses.replace(el, q=np.ascontiguousarray(el.q[:, :m])))
    ctx = cc.gpu_context(wl, options={cfft.OPT_DERIVATIVES: 1, cfft.OPT_FILL_TAPS: taps})
    ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP64, 4)
    pos = workloads.poisson_disc(60, 2.4, 0.4, seed=43)
    rot = workloads.rotations(len(pos), seed=43)
    a = len(pos)
    g = torch.tensor(workloads.complex_normal(a * m * a * m, 44).reshape(a * m, a * m), device="cuda:0")
    ref_p, ref_t = _adjoint(torch, ctx, pos, rot, g, -1)
    gp, gt = _adjoint(torch, ctx, pos, rot, g, 0)
    assert np.abs(gp - ref_p).max() < 1e-11 * np.abs(ref_p).max()
    assert np.all(np.abs(gt - ref_t) < 1e-11 * np.abs(ref_t))


def test_tensor_core_adjoint_vs_fp32_pipe(torch_cuda):
    """The adjoint of the tensor-core fill (forced: few pairs per cell here) against the
    bucketed adjoint on the FP32 pipe: position gradient (value and slope products, the
    q-weighted harmonics) and the substrate channels, 4 rotation classes, FP32."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch("fp32", n=1024, n_rho=1024, rho_max=9.0, q_max=4, rotation_classes=4)
    ctx = cc.gpu_context(wl, options={cfft.OPT_DERIVATIVES: 1})
    ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP32_MIXED, 4)
    pos = workloads.poisson_disc(300, 4.4, 0.3, seed=71)
    rot = workloads.rotations(len(pos), seed=71)
    a, m = len(pos), 4
    g = torch.tensor(workloads.complex_normal((a * m, a * m), 72), device="cuda:0").to(torch.complex64)
    ctx.set_option(cfft.OPT_FILL_SIMT, 1)
    ref_p, ref_t = _adjoint(torch, ctx, pos, rot, g, 0)
    ctx.set_option(cfft.OPT_FILL_SIMT, -1)
    gp, gt = _adjoint(torch, ctx, pos, rot, g, 0)
    ctx.set_option(cfft.OPT_FILL_SIMT, 0)
    ep = np.abs(gp - ref_p).max() / np.abs(ref_p).max()
    et = np.abs(gt - ref_t) / np.abs(ref_t)
    print("tensor-core adjoint vs FP32 pipe: pos", ep, "eps/h", et)
    assert ep < 2e-5 and np.all(et < 5e-5)
