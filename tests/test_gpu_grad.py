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
