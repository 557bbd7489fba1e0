"""GPU parity: the CUDA C-FFT tables and fills against the FP64 oracle.

Tolerances (relative to the table maximum of each (class, pair), as stated for
the tables): FP64 mode 1e-10, FP32-mixed mode 1e-5.  Stage buffers are
compared with their plain definitions (harmonics by an alpha trapezoid,
transform grid by the exact exponential sum).
"""
import math

import numpy as np
import pytest

import workloads
from tests import cfft_cases as cc
from oracle import reaction as orx

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_strip_fp64_full_table(torch_cuda):
    """Strip dipole, eps_r 2.2, h 0.05, N = 1024, 1024 rho to 10, |q| <= 4, complex128."""
    wl = workloads.strip_fp64()
    ctx, got = cc.gpu_table(wl)
    ref, nodes, hq = cc.oracle_table(wl)
    err = cc.rel_err_per_pair(got, ref)
    info = ctx.info()
    print("strip fp64 rel err", err.max(), info)
    assert err.max() < TOL["fp64"]


def test_strip_fp64_stages(torch_cuda):
    wl = workloads.strip_fp64(n=1024, n_rho=256, rho_max=10.0)
    ctx, got = cc.gpu_table(wl)
    nodes, hq = cc.oracle_harmonics(wl)
    # harmonics stage: H_q(beta_j) beta_j w_j
    y = ctx.debug_buffer("harmonics").cpu().numpy()[0]        # (pairs, nq, n)
    yref = (hq[0] * (nodes["beta_c"] * nodes["weight"])).reshape(y.shape)
    assert np.abs(y - yref).max() < 1e-12 * np.abs(yref).max()
    # grid stage: g_q(s_k) exp(i beta_max s_k / 2) against the exact exponential sum
    info = ctx.info()
    grid = ctx.debug_buffer("grid").cpu().numpy()[0]
    k = np.arange(-info["grid_half"], info["grid_half"] + 1)
    s = k * info["delta_s"]
    sel = np.abs(s) <= wl.rho_max
    e = np.exp(-1j * np.outer(nodes["beta_c"], s[sel]))
    gref = (yref @ e) * np.exp(1j * wl.contour.beta_max / 2 * s[sel])
    assert np.abs(grid[..., sel] - gref).max() < 1e-11 * np.abs(gref).max()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_patch_small_all_pairs(torch_cuda, precision):
    """Rooftop patch (200 rooftops, M = 4, 16 pairs) at a reduced contour/rho size."""
    wl = cc.small_patch(precision)
    ctx, got = cc.gpu_table(wl)
    ref, _, _ = cc.oracle_table(wl)
    err = cc.rel_err_per_pair(got, ref)
    print(precision, "patch rel err", err.max(), ctx.info())
    assert err.max() < TOL[precision]


def test_patch_rotation_classes(torch_cuda):
    wl = cc.small_patch("fp32", n=1024, n_rho=256, rho_max=4.0, q_max=3, rotation_classes=4)
    ctx, got = cc.gpu_table(wl)
    ref, _, _ = cc.oracle_table(wl, classes=(0, 1, 2, 3))
    err = cc.rel_err_per_pair(got, ref)
    print("rotation classes rel err", err.max(axis=1))
    assert err.max() < TOL["fp32"]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fill_small_array(torch_cuda, precision):
    torch = torch_cuda
    wl = cc.small_patch(precision, n=1024, n_rho=512, rho_max=5.0, q_max=4, rotation_classes=4)
    ctx, _ = cc.gpu_table(wl)
    pos = workloads.poisson_disc(24, 2.4, 0.5, seed=21)
    rot = workloads.rotations(24, seed=21)
    a = len(pos)
    m = wl.element.n_mbf
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    ld = a * m + 3  # a padded leading dimension
    z = torch.zeros((a * m, ld), dtype=dt, device="cuda:0")
    ctx.fill_reduced_matrix(torch.tensor(pos, device="cuda:0"),
                            torch.tensor(rot, device="cuda:0"), z)
    got = z.cpu().numpy()[:, :a * m]
    assert np.all(z.cpu().numpy()[:, a * m:] == 0)
    nodes, hq = cc.oracle_harmonics(wl, classes=(0, 1, 2, 3))
    pairs = [(i, j) for i in range(a) for j in range(a)]
    ref = cc.oracle_fill_entries(wl, hq, nodes, pos, rot, pairs)
    refm = np.zeros((a * m, a * m), dtype=np.complex128)
    for (i, j), blk in zip(pairs, ref):
        refm[i * m:(i + 1) * m, j * m:(j + 1) * m] = blk
    err = np.abs(got - refm).max() / np.abs(refm).max()
    print(precision, "fill rel err", err)
    assert err < TOL[precision]


def test_fill_host_variant_matches_device(torch_cuda):
    torch = torch_cuda
    wl = cc.small_patch("fp32", n=1024, n_rho=512, rho_max=5.0, q_max=2)
    ctx, _ = cc.gpu_table(wl)
    pos = workloads.poisson_disc(16, 2.0, 0.5, seed=5)
    a, m = len(pos), wl.element.n_mbf
    zd = torch.zeros((a * m, a * m), dtype=torch.complex64, device="cuda:0")
    ctx.fill_reduced_matrix(torch.tensor(pos, device="cuda:0"), None, zd)
    zh = np.zeros((a * m, a * m), dtype=np.complex64)
    ctx.fill_reduced_matrix_host(np.ascontiguousarray(pos), None, zh)
    assert np.array_equal(zd.cpu().numpy(), zh)


def test_fill_rejects_pairs_beyond_table(torch_cuda):
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch("fp32", n=1024, n_rho=256, rho_max=2.0, q_max=1)
    ctx, _ = cc.gpu_table(wl)
    pos = torch.tensor([[0.0, 0.0], [3.0, 0.0]], dtype=torch.float64, device="cuda:0")
    z = torch.zeros((8, 8), dtype=torch.complex64, device="cuda:0")
    with pytest.raises(cfft.CfftError) as ei:
        ctx.fill_reduced_matrix(pos, None, z)
    assert ei.value.status == 1


def test_state_machine_and_arguments(torch_cuda):
    from paper_1404_7357_gb300 import cfft
    ctx = cfft.Context(0)
    with pytest.raises(cfft.CfftError) as ei:
        ctx.build_contour(1024, 40.0, 12.0, 0.2)
    assert ei.value.status == 2
    ctx.set_substrate(2.2, 0.05, 2 * math.pi)
    with pytest.raises(cfft.CfftError) as ei:
        ctx.tabulate_reactions(2, 5.0, 64, cfft.CFFT_FP64)
    assert ei.value.status == 2
    with pytest.raises(cfft.CfftError) as ei:
        ctx.build_contour(1024, 40.0, 5.0, 0.2)   # beta_p below k_d: poles not enclosed
    assert ei.value.status == 1
    with pytest.raises(cfft.CfftError) as ei:
        ctx.set_substrate(-1.0, 0.05, 2 * math.pi)
    assert ei.value.status == 1
    with pytest.raises(cfft.CfftError):
        ctx.get_table()


def test_degenerate_q0_and_tiny_grid(torch_cuda):
    """q_max = 0 (a single harmonic) and the smallest contour the library accepts."""
    wl = workloads.strip_fp64(n=64, n_rho=40, rho_max=1.0, q_max=0)
    ctx, got = cc.gpu_table(wl)
    ref, _, _ = cc.oracle_table(wl)
    assert cc.rel_err_per_pair(got, ref).max() < TOL["fp64"]


def test_taylor_order_trend(torch_cuda):
    """Error falls with the Taylor order (the trend of the paper's Table I)."""
    errs = []
    for nt in (0, 1, 2, 3, 6):
        wl = workloads.strip_fp64(n=1024, n_rho=128, rho_max=10.0)
        wl.extras["taylor"] = nt
        _, got = cc.gpu_table(wl)
        if nt == 0:
            ref, _, _ = cc.oracle_table(wl)
        errs.append(cc.rel_err_per_pair(got, ref).max())
    print("taylor trend", errs)
    assert all(b < a for a, b in zip(errs, errs[1:]))


@pytest.mark.slow
def test_patch_full_size_sampled(torch_cuda):
    """Full-size patch table (N = 16384, 8192 rho to 50, |q| <= 16, 16 pairs), FP32-mixed,
    checked on sampled rho rows for every pair and harmonic."""
    wl = workloads.patch_m4()
    ctx, got = cc.gpu_table(wl)
    rows = np.array([0, 1, 7, 333, 2048, 4097, 6000, 8191])
    ref, _, _ = cc.oracle_table(wl, rho_index=rows)
    err = cc.rel_err_per_pair(got[..., rows], ref)
    print("full-size sampled rel err", err.max(), ctx.info())
    assert err.max() < TOL["fp32"]


@pytest.mark.slow
def test_patch_full_size_fp64_sampled(torch_cuda):
    """The same full-size patch table in the plain FP64 form (zero padding 8, 16-tap
    stencils, Taylor order for 1e-13), against the oracle at the 1e-10 target on sampled
    rho rows for every pair and harmonic -- up to rho = 50 wavelengths, where the angular
    quadrature of the back-projection needs the most nodes."""
    wl = workloads.patch_m4(precision="fp64")
    ctx, got = cc.gpu_table(wl)
    rows = np.array([0, 1, 7, 333, 2048, 4097, 6000, 7500, 8191])
    ref, _, _ = cc.oracle_table(wl, rho_index=rows)
    err = cc.rel_err_per_pair(got[..., rows], ref)
    # per sampled row, so that a failure shows where in rho it lies
    per_row = (np.abs(got[..., rows] - ref).max(axis=(0, 1, 2)) /
               np.abs(ref).reshape(-1, len(rows)).max())
    print("full-size FP64 sampled rel err", err.max(), "by row", dict(zip(rows.tolist(), per_row)))
    assert err.max() < TOL["fp64"]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_backprojection_forms_agree(torch_cuda, precision):
    """The matrix form and the direct gather form of the back-projection evaluate the
    same quadrature; both against the oracle (3 rotation classes: 48 series per q)."""
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch(precision, n=1024, n_rho=200, rho_max=4.0, q_max=2, rotation_classes=4)
    _, w_form = cc.gpu_table(wl)
    _, g_form = cc.gpu_table(wl, options={cfft.OPT_BP_GATHER: 1})
    ref, _, _ = cc.oracle_table(wl, classes=(0, 1, 2, 3))
    ew = cc.rel_err_per_pair(w_form, ref).max()
    eg = cc.rel_err_per_pair(g_form, ref).max()
    print(precision, "matrix form", ew, "gather form", eg)
    assert ew < TOL[precision] and eg < TOL[precision]


def test_fp32_single_harmonic_and_ragged_tiles(torch_cuda):
    """FP32-mixed with q_max = 0 (the paired-harmonic back-projection with |q| = 0 only)
    and a rho grid that ends inside a row tile."""
    wl = cc.small_patch("fp32", n=1024, n_rho=300, rho_max=4.0, q_max=0)
    ctx, got = cc.gpu_table(wl)
    ref, _, _ = cc.oracle_table(wl)
    err = cc.rel_err_per_pair(got, ref).max()
    print("fp32 q_max=0 rel err", err)
    assert err < TOL["fp32"]


@pytest.mark.parametrize("taps,kern", [(8, 1), (12, 1), (16, 1), (6, 2), (8, 2)])
def test_backprojection_tensor_cores_vs_fp32_pipe(torch_cuda, taps, kern):
    """The paired-harmonic back-projection with its products on the tensor cores (three
    TF32 products per K-tile, drained into FP32 registers) against the same form on the
    FP32 pipe and against the oracle: 3 computed rotation classes (48 series per q, three
    series chunks), a ragged last row tile, many K-tiles, each stencil width, Lagrange
    (kern 1) and ES (kern 2) stencils."""
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch("fp32", n=2048, n_rho=600, rho_max=9.0, q_max=3, rotation_classes=4)
    opts = {cfft.OPT_BP_TAPS: taps, cfft.OPT_BP_KERNEL: kern}
    ctx_t, t_form = cc.gpu_table(wl, options=opts)
    ctx_s, s_form = cc.gpu_table(wl, options={**opts, cfft.OPT_BP_SIMT: 1})
    assert ctx_t.info()["bp_form"] == 3 and ctx_s.info()["bp_form"] == 2
    assert ctx_t.info()["bp_kernel"] == kern - 1 and ctx_s.info()["bp_kernel"] == kern - 1
    ref, _, _ = cc.oracle_table(wl, classes=(0, 1, 2, 3))
    et = cc.rel_err_per_pair(t_form, ref).max()
    es = cc.rel_err_per_pair(s_form, ref).max()
    ets = cc.rel_err_per_pair(t_form, s_form.astype(np.complex128)).max()
    print("taps", taps, "kernel", kern, "tensor-core form", et, "FP32-pipe form", es, "between", ets)
    assert ets < 2e-6
    if taps >= 12 or kern == 2:   # 8 Lagrange taps are below the FP32 target on this grid
        assert et < TOL["fp32"] and es < TOL["fp32"]
