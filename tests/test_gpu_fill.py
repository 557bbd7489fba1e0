"""The bucketed fill (pairs counting-sorted by class and stencil row, table windows in
shared memory) against the per-row fill and the oracle, over the cases it covers:
M in {1, 2, 4}, 8/12/16 taps, several row-block sizes (blocks that split the element
set raggedly), padded and odd leading dimensions, and pairs on the parity rows."""
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


def _fill(torch, ctx, pos, rot, m, dt, ld=None, block=None):
    from paper_1404_7357_gb300 import cfft
    a = len(pos)
    ld = ld or a * m
    if block is not None:
        ctx.set_option(cfft.OPT_FILL_BLOCK, block)
    z = torch.full((a * m, ld), 7.0, dtype=dt, device="cuda:0")
    rt = None if rot is None else torch.tensor(rot, device="cuda:0")
    ctx.fill_reduced_matrix(torch.tensor(pos, device="cuda:0"), rt, z)
    out = z.cpu().numpy()
    assert np.all(out[:, a * m:] == 7.0)   # padding untouched
    return out[:, :a * m]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_bucketed_matches_per_row(torch_cuda, precision):
    torch = torch_cuda
    wl = cc.small_patch(precision, n=1024, n_rho=1024, rho_max=9.0, q_max=4, rotation_classes=4)
    ctx, _ = cc.gpu_table(wl)
    pos = workloads.poisson_disc(300, 4.4, 0.3, seed=31)
    rot = workloads.rotations(len(pos), seed=31)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    ref = _fill(torch, ctx, pos, rot, 4, dt, block=-1)
    tol = 1e-12 if precision == "fp64" else 2e-6
    scale = np.abs(ref).max()
    for block in (0, 5, 37, 1000):
        got = _fill(torch, ctx, pos, rot, 4, dt, block=block)
        err = np.abs(got - ref).max() / scale
        print(precision, "block", block, "bucketed vs per-row", err)
        assert err < tol


@pytest.mark.parametrize("ld_pad", [0, 1, 2])
def test_bucketed_leading_dimensions(torch_cuda, ld_pad):
    torch = torch_cuda
    wl = cc.small_patch("fp32", n=1024, n_rho=512, rho_max=5.0, q_max=3)
    ctx, _ = cc.gpu_table(wl)
    pos = workloads.poisson_disc(40, 2.4, 0.5, seed=7)
    a = len(pos)
    ref = _fill(torch, ctx, pos, None, 4, torch.complex64, block=-1)
    got = _fill(torch, ctx, pos, None, 4, torch.complex64, ld=a * 4 + ld_pad, block=0)
    assert np.abs(got - ref).max() < 2e-6 * np.abs(ref).max()


@pytest.mark.parametrize("taps", [8, 12, 16])
def test_bucketed_taps_and_m2(torch_cuda, taps):
    """M = 2 (two MBFs from the rooftop set) and each templated stencil width."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch("fp32", n=1024, n_rho=512, rho_max=5.0, q_max=2, rotation_classes=4)
    el = wl.element
    wl = dataclasses.replace(wl, element=dataclasses.replace(el, q=np.ascontiguousarray(el.q[:, :2])))
    ctx = cc.gpu_context(wl, options={cfft.OPT_FILL_TAPS: taps})
    ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP32_MIXED, 4)
    pos = workloads.poisson_disc(40, 2.4, 0.5, seed=8)
    rot = workloads.rotations(len(pos), seed=8)
    ref = _fill(torch, ctx, pos, rot, 2, torch.complex64, block=-1)
    got = _fill(torch, ctx, pos, rot, 2, torch.complex64, block=0)
    assert np.abs(got - ref).max() < 2e-6 * np.abs(ref).max()


def test_bucketed_strip_m1_against_oracle(torch_cuda):
    """M = 1 (strip dipole, FP64) against the oracle, including pairs closer than one
    stencil half-width to rho = 0 (parity rows) and the diagonal."""
    torch = torch_cuda
    wl = workloads.strip_fp64(n=1024, n_rho=512, rho_max=4.0, q_max=4)
    ctx, _ = cc.gpu_table(wl)
    rng = np.random.default_rng(3)
    pos = np.concatenate([rng.uniform(-1.3, 1.3, (18, 2)),
                          np.array([[0.0, 0.0], [0.004, 0.003], [-0.002, 0.01]])])
    got = _fill(torch, ctx, pos, None, 1, torch.complex128, block=0)
    nodes, hq = cc.oracle_harmonics(wl)
    a = len(pos)
    pairs = [(i, j) for i in range(a) for j in range(a)]
    rot0 = np.zeros(a, dtype=np.int32)
    ref = np.array([blk[0, 0] for blk in cc.oracle_fill_entries(wl, hq, nodes, pos, rot0, pairs)])
    err = np.abs(got.reshape(-1) - ref).max() / np.abs(ref).max()
    print("strip M=1 bucketed vs oracle", err)
    assert err < 1e-10


@pytest.mark.parametrize("block", [0, 37])
def test_tensor_core_fill_vs_fp32_pipe(torch_cuda, block):
    """The fill of M = 4 with 8 taps as one tensor-core contraction per stencil cell
    (three TF32 products) against the bucketed fill on the FP32 pipe and the oracle's
    exact entries: 4 rotation classes, pairs near rho = 0 (parity rows), one row block
    (block 0) and ragged row blocks (37)."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch("fp32", n=1024, n_rho=1024, rho_max=9.0, q_max=4, rotation_classes=4)
    ctx, _ = cc.gpu_table(wl)
    pos = np.concatenate([workloads.poisson_disc(300, 4.4, 0.3, seed=61), [[0.01, -0.02], [0.012, -0.019]]])
    rot = workloads.rotations(len(pos), seed=61)
    ref = _fill(torch, ctx, pos, rot, 4, torch.complex64, block=block)                 # default: tensor cores
    ctx.set_option(cfft.OPT_FILL_SIMT, 1)
    simt = _fill(torch, ctx, pos, rot, 4, torch.complex64, block=block)
    ctx.set_option(cfft.OPT_FILL_SIMT, 0)
    scale = np.abs(simt).max()
    err = np.abs(ref - simt).max() / scale
    print("block", block, "tensor-core fill vs FP32-pipe fill", err)
    assert err < 5e-6
    # a sample of entries against the oracle's exact fill
    nodes, hq = cc.oracle_harmonics(wl, classes=(0, 1, 2, 3))
    idx = [(0, 1), (5, 300), (300, 301), (17, 17), (120, 44)]
    exact = cc.oracle_fill_entries(wl, hq, nodes, pos, rot, idx)
    for (i, j), blk in zip(idx, exact):
        got = ref[4 * i:4 * i + 4, 4 * j:4 * j + 4]
        assert np.abs(got - blk).max() < 1e-5 * scale, (i, j)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_table_checkpoint_and_resume(torch_cuda, tmp_path, precision):
    """save_table / load_table (cfft_load_table): a fresh context with no substrate,
    element or contour fills from the saved table exactly as the tabulating one does."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch(precision, n=1024, n_rho=1024, rho_max=5.0, q_max=3, rotation_classes=4)
    ctx, _ = cc.gpu_table(wl)
    pos = workloads.poisson_disc(40, 2.4, 0.5, seed=81)
    rot = workloads.rotations(len(pos), seed=81)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    ref = _fill(torch, ctx, pos, rot, 4, dt)
    # this grid meets the fill's target as tabulated: the fill used the saved table itself
    assert ctx.info()["fill_refine"] == 1 and ctx.info()["fill_n_rho"] == wl.n_rho
    desc = ctx.save_table(str(tmp_path / "table"))
    fresh = cfft.Context(0)
    got_desc = fresh.load_table(str(tmp_path / "table"))
    assert got_desc == desc
    got = _fill(torch, fresh, pos, rot, 4, dt)
    assert np.array_equal(got, ref)
    # a description that does not fit is refused
    with pytest.raises(cfft.CfftError):
        fresh._check(cfft._lib.cfft_load_table(fresh._h, 4, 3, 5.0, 10, 0, 4, 8, None, 1))


def _line_array():
    """Elements on a line whose pair distances run from 0.03 to 2.97 wavelengths: the short
    ones where the table varies fastest, the long ones within half a stencil of rho_max."""
    x = np.array([0.0, 0.031, 0.077, 0.52, 1.5, 2.97])
    return np.stack([x, 0.37 * x], 1) / np.hypot(1.0, 0.37)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fill_meets_target_at_every_distance(torch_cuda, precision):
    """The table grid here (256 rho points to 3 wavelengths) is too coarse for the fill's
    Lagrange stencil at short distances and next to rho_max.  The library estimates the
    interpolation error from the table's p-th differences, finds it above the precision's
    share, and tabulates the fill's own table on a finer grid reaching past rho_max: every
    entry then meets the target against the oracle's exact fill.  Forcing the tabulated grid
    (FILL_REFINE = 1) shows the error the refinement removes, and that the estimate is not
    below it."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch(precision, n=1024, n_rho=256, rho_max=3.0, q_max=2)
    ctx, _ = cc.gpu_table(wl)
    pos = _line_array()
    a, m = len(pos), 4
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    nodes, hq = cc.oracle_harmonics(wl)
    pairs = [(i, j) for i in range(a) for j in range(a)]
    blocks = cc.oracle_fill_entries(wl, hq, nodes, pos, np.zeros(a, dtype=np.int32), pairs)
    zref = np.zeros((a * m, a * m), dtype=np.complex128)
    for (i, j), blk in zip(pairs, blocks):
        zref[i * m:(i + 1) * m, j * m:(j + 1) * m] = blk
    scale = np.abs(zref).max()
    got = _fill(torch, ctx, pos, None, m, dt)
    info = ctx.info()
    err = np.abs(got - zref).max() / scale
    ctx.set_option(cfft.OPT_FILL_REFINE, 1)
    coarse = _fill(torch, ctx, pos, None, m, dt)
    err_coarse = np.abs(coarse - zref).max() / scale
    print(precision, "estimate on the tabulated grid %.3g, refine %d, fill grid %d: error %.3g; on the "
          "tabulated grid %.3g" % (info["fill_err_est"], info["fill_refine"], info["fill_n_rho"], err,
                                    err_coarse))
    share = 0.25 * TOL[precision]
    assert info["fill_err_est"] > share and info["fill_n_rho"] > wl.n_rho
    assert info["fill_n_rho"] == (wl.n_rho - 1) * info["fill_refine"] + 1 + info["fill_taps"] // 2
    assert err < TOL[precision]
    assert err_coarse > err and err_coarse < 2.0 * info["fill_err_est"]


def test_loaded_coarse_table_is_refused(torch_cuda, tmp_path):
    """A loaded table cannot be tabulated again: a fill on a grid that misses the target is
    refused (CFFT_ERR_ARG) instead of returning a less accurate matrix; FILL_REFINE = 1 then
    fills on that grid, exactly as the tabulating context does with the same setting."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch("fp64", n=1024, n_rho=256, rho_max=3.0, q_max=2)
    ctx, _ = cc.gpu_table(wl)
    ctx.set_option(cfft.OPT_FILL_REFINE, 1)
    pos = _line_array()
    ref = _fill(torch, ctx, pos, None, 4, torch.complex128)
    ctx.save_table(str(tmp_path / "coarse"))
    fresh = cfft.Context(0)
    fresh.load_table(str(tmp_path / "coarse"))
    z = torch.zeros((len(pos) * 4, len(pos) * 4), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(cfft.CfftError) as ei:
        fresh.fill_reduced_matrix(torch.tensor(pos, device="cuda:0"), None, z)
    assert ei.value.status == 1
    fresh.set_option(cfft.OPT_FILL_REFINE, 1)
    got = _fill(torch, fresh, pos, None, 4, torch.complex128)
    assert np.array_equal(got, ref)


@pytest.mark.slow
def test_full_size_fill_sampled_against_oracle(torch_cuda):
    """The benchmark's fill at full size and in its launch configuration (10,000-element
    irregular array, 40,000^2 complex64, table of patch-m4 with 4 rotation classes to
    121 lambda0 on 16,384 points, FP32-mixed, tensor-core form): sampled element-pair
    blocks (near, middle and far pairs, every rotation class, a diagonal block) against
    the oracle's exact fill on the same contour."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = workloads.patch_m4(n=16384, n_rho=16384, rho_max=121.0, q_max=16, precision="fp32",
                            rotation_classes=4)
    pos, rot = workloads.irregular_array()
    ctx, _ = cc.gpu_table(wl)
    a, m = len(pos), 4
    z = torch.empty((a * m, a * m), dtype=torch.complex64, device="cuda:0")
    ctx.fill_reduced_matrix(torch.tensor(pos, device="cuda:0"), torch.tensor(rot, device="cuda:0"), z)
    assert ctx.info()["fill_form"] == 3
    rng = np.random.default_rng(91)
    d = np.hypot(*(pos[:, None, :] - pos[None, :10, :]).transpose(2, 0, 1))   # to 10 anchors
    pairs = [(0, 0)]
    for lo, hi in ((0.4, 2.0), (20.0, 40.0), (60.0, 80.0), (100.0, 121.0)):
        cand = np.argwhere((d >= lo) & (d < hi))
        for k in rng.choice(len(cand), size=min(4, len(cand)), replace=False):
            pairs.append((int(cand[k][0]), int(cand[k][1])))
    got = [z[4 * i:4 * i + 4, 4 * j:4 * j + 4].cpu().numpy().astype(np.complex128) for i, j in pairs]
    del z
    torch.cuda.empty_cache()
    nodes, hq = cc.oracle_harmonics(wl, classes=(0, 1, 2, 3))
    ref = cc.oracle_fill_entries(wl, hq, nodes, pos, rot, pairs)
    scale = max(np.abs(r).max() for r in ref)
    err = max(np.abs(g - r).max() for g, r in zip(got, ref)) / scale
    classes = {2 * int(rot[i]) + int(rot[j]) for i, j in pairs}
    print("full-size fill, %d sampled blocks (classes %s): rel err %.3g" % (len(pairs), sorted(classes), err))
    assert err < 1e-5
