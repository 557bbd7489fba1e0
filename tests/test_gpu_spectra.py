"""MBF spectra on the tensor cores (cfft_mbf_spectra) against the oracle's Eq. 11.

FP32 operands with TF32 head/tail splitting must reproduce float32 accuracy:
relative to the largest spectrum magnitude, 1e-5 (the FP32-mixed tolerance of the
tables).  Cases: contour-like wavevectors beta_c (cos, sin)(alpha), arbitrary complex
wavevectors, M = 1, 2, 4 (the compiled column layouts), several rooftop shapes
(more GEMM columns), a point count that is not a multiple of the 128-row tile, and
more tiles than SMs (the persistent tile loop)."""
import dataclasses

import numpy as np
import pytest

import workloads
from tests import cfft_cases as cc
from oracle import spectra as osp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _ctx(el):
    from paper_1404_7357_gb300 import cfft
    ctx = cfft.Context(0)
    ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
    return ctx


def _points(n, seed, beta_max=66.0, height=0.03):
    """Half contour-like, half arbitrary complex wavevectors."""
    rng = np.random.default_rng(seed)
    m = n // 2
    br = rng.uniform(0.0, beta_max, m)
    bi = height * rng.uniform(0.0, 1.0, m)
    al = rng.uniform(0.0, 2 * np.pi, m)
    b = br + 1j * bi
    kx1, ky1 = b * np.cos(al), b * np.sin(al)
    kx2 = rng.normal(0, 20, n - m) + 1j * rng.normal(0, 0.5, n - m)
    ky2 = rng.normal(0, 20, n - m) + 1j * rng.normal(0, 0.5, n - m)
    return np.concatenate([kx1, kx2]), np.concatenate([ky1, ky2])


def _check(torch, el, n, seed, tol=1e-5):
    ctx = _ctx(el)
    kx, ky = _points(n, seed)
    k = torch.tensor(np.stack([kx, ky], 1).astype(np.complex64), device="cuda:0")
    got = ctx.mbf_spectra(k).cpu().numpy().astype(np.complex128)    # (n, 2, M, 2)
    bs = cc.oracle_basis(el)
    kx64 = k.cpu().numpy()[:, 0].astype(np.complex128)               # the points as the GPU saw them
    ky64 = k.cpu().numpy()[:, 1].astype(np.complex128)
    err = 0.0
    scale = 0.0
    for side, conj in ((0, False), (1, True)):
        mx, my = osp.mbf_spectra(bs, kx64, ky64, conjugate_side=conj)   # (M, n) each
        ref = np.stack([mx.T, my.T], -1)                                  # (n, M, 2)
        err = max(err, np.abs(got[:, side] - ref).max())
        scale = max(scale, np.abs(ref).max())
    print("spectra M=%d n=%d rel err %.3g" % (el.n_mbf, n, err / scale))
    assert err / scale < tol


@pytest.mark.parametrize("m", [1, 2, 4])
def test_spectra_patch(torch_cuda, m):
    el = workloads.patch_rooftops()
    el = dataclasses.replace(el, q=np.ascontiguousarray(el.q[:, :m]))
    _check(torch_cuda, el, 1000, seed=m)


def test_spectra_mixed_shapes_and_many_tiles(torch_cuda):
    """Four rooftop shapes (two sizes per direction): 64 GEMM columns; 39,000 points
    (305 tiles of 128, more than one per SM)."""
    el = workloads.patch_rooftops()
    hl = el.half_len.copy()
    hl[::3] *= 1.5
    el = dataclasses.replace(el, half_len=hl)
    _check(torch_cuda, el, 39000, seed=7)


def test_spectra_rejects_strip(torch_cuda):
    from paper_1404_7357_gb300 import cfft
    torch = torch_cuda
    ctx = cfft.Context(0)
    ctx.set_mbf_spectra_strip(0.45, 0.02)
    k = torch.zeros((4, 2), dtype=torch.complex64, device="cuda:0")
    with pytest.raises(cfft.CfftError) as ei:
        ctx.mbf_spectra(k)
    assert ei.value.status == 1


@pytest.mark.parametrize("n_alpha", [128, 256])
def test_integrand_tensor_cores_vs_simt_and_oracle(torch_cuda, n_alpha):
    """The FP32-mixed tabulation with the spectra on the tensor cores (default) and with
    SIMT spectra: contour harmonics Y = H_ab,q beta_c w against the oracle's, and tables,
    for 128 and 256 angles (angular folds 4 and 8)."""
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch("fp32", n=1024, n_rho=256, rho_max=4.0, q_max=4)
    nodes, hq = cc.oracle_harmonics(wl)
    ref_tab, _, _ = cc.oracle_table(wl)
    out = {}
    for name, opts in (("tensor", {cfft.OPT_N_ALPHA: n_alpha}),
                       ("simt", {cfft.OPT_N_ALPHA: n_alpha, cfft.OPT_SPECTRA_SIMT: 1})):
        ctx, tab = cc.gpu_table(wl, options=opts)
        assert ctx.info()["spectra_tc"] == (1 if name == "tensor" else 0)
        y = ctx.debug_buffer("harmonics").cpu().numpy()[0].astype(np.complex128)
        yref = (hq[0] * (nodes["beta_c"] * nodes["weight"])).reshape(y.shape)
        ey = np.abs(y - yref).max() / np.abs(yref).max()
        et = cc.rel_err_per_pair(tab, ref_tab).max()
        out[name] = (ey, et)
        print(name, n_alpha, "harmonics rel err %.3g, table rel err %.3g" % (ey, et))
        assert ey < 1e-5 and et < 1e-5


def test_spectra_small_complex_wavevectors(torch_cuda):
    """Small complex k (|k a / 2| ~ 0.01 with a small imaginary part): the rooftop factor
    sinc(z) there is sensitive to how sinh(Im z) is formed."""
    torch = torch_cuda
    el = workloads.patch_rooftops()
    ctx = _ctx(el)
    rng = np.random.default_rng(5)
    n = 2000
    b = rng.uniform(0.2, 1.0, n) + 1j * rng.uniform(1e-4, 0.01, n)
    al = rng.uniform(0, 2 * np.pi, n)
    k = torch.tensor(np.stack([b * np.cos(al), b * np.sin(al)], 1).astype(np.complex64), device="cuda:0")
    got = ctx.mbf_spectra(k).cpu().numpy().astype(np.complex128)
    kk = k.cpu().numpy().astype(np.complex128)
    bs = cc.oracle_basis(el)
    mx, my = osp.mbf_spectra(bs, kk[:, 0], kk[:, 1])
    ref = np.stack([mx.T, my.T], -1)
    err = np.abs(got[:, 0] - ref).max() / np.abs(ref).max()
    print("small complex k rel err %.3g" % err)
    assert err < 3e-6
