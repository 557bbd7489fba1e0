"""GPU cases for configurations and failure paths beyond the per-stage files: the batched
sweep's graph capture and recapture, the strip element in batches and in FP32-mixed, the
benchmarked sweep at full size, eight MBFs, the smallest arrays, the residual form of
the fill adjoint, out-of-memory injected on the host, and empty inputs.  Every case runs through the
C ABI and is compared with the oracle or with a path checked against it.  Nothing here
traps, faults or waits without a bound."""
import numpy as np
import pytest

import workloads
from tests import cfft_cases as cc
from tests.test_gpu_batch import _items, _single

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_batch_graph_replayed_on_new_substrates(torch_cuda):
    """Same structure, new substrates: the second call replays the captured graph (the
    context's capture count stays at one) and the tables follow the new parameters."""
    from paper_1404_7357_gb300 import cfft
    el = workloads.patch_rooftops()
    items = _items(4, seed=11)
    q_max, rho_max, n_rho = 2, 3.0, 128
    ctx = cfft.Context(0)
    ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
    ctx.set_option(cfft.OPT_N_ALPHA, 128)
    out = ctx.tabulate_batch(items, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, graph=True)
    first = out.cpu().numpy().copy()
    assert ctx.batch_info()["captures"] == 1
    for it in items:
        it["h"] *= 1.1
    out = ctx.tabulate_batch(items, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, out=out, graph=True)
    assert ctx.batch_info()["captures"] == 1          # replayed, not captured again
    assert np.abs(out.cpu().numpy() - first).max() > 1e-3 * np.abs(first).max()


def test_batch_graph_recaptured_when_the_contours_change(torch_cuda):
    """Same item count, node counts and Taylor orders, new contours: beta_max, the pole
    bound and the height move, so the transform grids and the angular node counts change.
    The captured graph holds those shapes and buffer addresses, so it must not be replayed
    on the new plan: it is captured again, and the tables match single tabulations."""
    from paper_1404_7357_gb300 import cfft
    el = workloads.patch_rooftops()
    items = _items(4, seed=11)
    for it in items:
        it["taylor_order"] = 26   # fixed, so only the contour geometry changes below
    q_max, rho_max, n_rho = 2, 3.0, 128
    ctx = cfft.Context(0)
    ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
    ctx.set_option(cfft.OPT_N_ALPHA, 128)
    out = ctx.tabulate_batch(items, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, graph=True)
    assert ctx.batch_info()["captures"] == 1
    for it in items:
        kd = it["k0"] * np.sqrt(it["eps_r"])
        it["beta_max"] = 5.25 * kd
        step = it["beta_max"] / it["n"]
        it["beta_p"] = round(1.3 * kd / step) * step
        it["height"] = 6.0 * step
    out = ctx.tabulate_batch(items, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, out=out, graph=True)
    assert ctx.batch_info()["captures"] == 2      # the plan moved: captured again
    got = out.cpu().numpy()
    for i, it in enumerate(items):
        ref = _single(cfft, el, it, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, 128)
        err = np.abs(got[i].astype(np.complex128) - ref).max() / np.abs(ref).max()
        print("item", i, "n", it["n"], "rel err after the contour change", err)
        assert err < TOL["fp32"]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_strip_matches_single_tabulations(torch_cuda, precision):
    """A batch of the strip element (M = 1: one series per harmonic, SIMT spectra) against
    single tabulations of the same items."""
    from paper_1404_7357_gb300 import cfft
    prec = cfft.CFFT_FP64 if precision == "fp64" else cfft.CFFT_FP32_MIXED
    el = workloads.strip_element()
    items = _items(3, seed=17)
    q_max, rho_max, n_rho = 3, 3.0, 200
    ctx = cfft.Context(0)
    ctx.set_mbf_spectra_strip(el.length, el.strip_width)
    ctx.set_option(cfft.OPT_N_ALPHA, 128)
    got = ctx.tabulate_batch(items, q_max, rho_max, n_rho, prec, graph=True).cpu().numpy()
    for i, it in enumerate(items):
        one = cfft.Context(0)
        one.set_substrate(it["eps_r"], it["h"], it["k0"])
        one.set_mbf_spectra_strip(el.length, el.strip_width)
        one.build_contour(it["n"], it["beta_max"], it["beta_p"], it["height"], -1)
        one.set_option(cfft.OPT_N_ALPHA, 128)
        one.tabulate_reactions(q_max, rho_max, n_rho, prec, 1)
        ref = one.copy_table(host=True).numpy()[0]
        err = np.abs(got[i].astype(np.complex128) - ref).max() / np.abs(ref).max()
        print(precision, "strip batch item", i, "rel err vs single", err)
        assert err < TOL[precision]


@pytest.mark.slow
def test_full_size_sweep_sampled_against_oracle(torch_cuda):
    """The benchmarked sweep at full size -- 512 items (64 frequencies x 8 substrates),
    contours of 4k..64k nodes, M = 4, |q| <= 16, 2048 rho points to 50 lambda0, FP32-mixed,
    autotuned and replayed from one CUDA graph -- checked against the oracle on sampled
    rho rows (every pair and harmonic) of three items: the coarsest contour whose height
    sits at the cap height * rho_max = 3 (the fewest node spacings high), the largest
    beta_max, and a low contour."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    items = workloads.sweep_items()
    q_max, rho_max, n_rho = 16, 50.0, 2048
    el = workloads.patch_rooftops()
    ctx = cfft.Context(0)
    ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
    out = torch.empty((len(items), 16, 2 * q_max + 1, n_rho), dtype=torch.complex64, device="cuda:0")
    ctx.tabulate_batch(items, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, out=out, graph=True, autotune=True)
    ctx.tabulate_batch(items, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, out=out, graph=True)  # replay
    print("sweep batch info", ctx.batch_info())
    x = np.array([it["height"] * rho_max for it in items])
    ns = np.array([it["n"] for it in items])
    bmax = np.array([it["beta_max"] for it in items])
    small = ns <= 16384                              # keeps the oracle's share to seconds
    capped = np.flatnonzero(small & (x > 3.0 - 1e-9))
    picks = [int(capped[np.argmax(bmax[capped] / ns[capped])]),     # fewest node spacings high
             int(np.flatnonzero(small)[np.argmax(bmax[small])]),
             int(np.flatnonzero(small)[np.argmin(x[small])])]
    rows = np.array([0, 1, 511, 1024, 1800, 2047])
    for i in picks:
        it = items[i]
        wl = workloads.TableWorkload("sweep-item", workloads.Substrate(it["eps_r"], it["h"], it["k0"]), el,
                                     workloads.ContourSpec(it["n"], it["beta_max"], it["beta_p"], it["height"]),
                                     q_max, rho_max, n_rho, "fp32")
        got = out[i].cpu().numpy()[..., rows][None]
        ref, _, _ = cc.oracle_table(wl, rho_index=rows)
        err = cc.rel_err_per_pair(got, ref).max()
        print("sweep item %d: n %d beta_max %.1f height*rho_max %.2f  rel err %.2e" % (
            i, it["n"], it["beta_max"], x[i], err))
        assert err < TOL["fp32"]


@pytest.mark.parametrize("bp_simt", [0, 1])
def test_strip_fp32_single_series(torch_cuda, bp_simt):
    """The strip (M = 1) in FP32-mixed: one series per harmonic, so the back-projection's
    16-series chunk is mostly empty (tensor-core products and FP32-pipe products), and
    the SIMT spectra of a non-rooftop element; the whole table against the oracle."""
    import dataclasses
    from paper_1404_7357_gb300 import cfft
    wl = dataclasses.replace(workloads.strip_fp64(n=1024, n_rho=512, rho_max=8.0), precision="fp32")
    ctx, got = cc.gpu_table(wl, options={cfft.OPT_BP_SIMT: bp_simt})
    ref, _, _ = cc.oracle_table(wl)
    err = cc.rel_err_per_pair(got, ref).max()
    info = ctx.info()
    print("strip fp32 bp_simt", bp_simt, "bp form", info["bp_form"], "rel err", err)
    assert info["bp_form"] == (2 if bp_simt else 3)
    assert err < TOL["fp32"]


@pytest.fixture(scope="module")
def small_array_oracle():
    """Oracle harmonics of the small patch table used by the smallest-array fills (FP64
    definitions, the same for both GPU precisions), computed once for the module."""
    wl = cc.small_patch("fp64", n=1024, n_rho=512, rho_max=5.0, q_max=4, rotation_classes=4)
    return cc.oracle_harmonics(wl, classes=(0, 1, 2, 3))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", ["one", "two", "three"])
def test_fill_smallest_arrays(torch_cuda, small_array_oracle, precision, case):
    """Degenerate arrays: one element (its self block only, rho = 0), two and three
    elements with mixed rotations; every entry against the oracle's exact fill (FP32:
    the tensor-core form, one stencil cell per CTA and a ragged tile of pairs)."""
    torch = torch_cuda
    pos, rot = {"one": ([[0.3, -0.2]], [1]),
                "two": ([[0.0, 0.0], [1.7, 2.1]], [0, 1]),
                "three": ([[0.0, 0.0], [0.6, 0.0], [-2.0, 3.5]], [1, 0, 1])}[case]
    pos, rot = np.array(pos, dtype=np.float64), np.array(rot, dtype=np.int32)
    wl = cc.small_patch(precision, n=1024, n_rho=512, rho_max=5.0, q_max=4, rotation_classes=4)
    ctx, _ = cc.gpu_table(wl)
    a, m = len(pos), wl.element.n_mbf
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    z = torch.full((a * m, a * m), complex(float("nan"), 0.0), dtype=dt, device="cuda:0")
    ctx.fill_reduced_matrix(torch.tensor(pos, device="cuda:0"), torch.tensor(rot, device="cuda:0"), z)
    got = z.cpu().numpy()
    assert np.isfinite(got).all()          # every entry written
    nodes, hq = small_array_oracle
    pairs = [(i, j) for i in range(a) for j in range(a)]
    ref = cc.oracle_fill_entries(wl, hq, nodes, pos, rot, pairs)
    refm = np.zeros((a * m, a * m), dtype=np.complex128)
    for (i, j), blk in zip(pairs, ref):
        refm[i * m:(i + 1) * m, j * m:(j + 1) * m] = blk
    err = np.abs(got - refm).max() / np.abs(refm).max()
    print(precision, case, "fill form", ctx.info()["fill_form"], "rel err", err)
    assert err < TOL[precision]


def _eight_mbf_patch(precision):
    import dataclasses
    wl = cc.small_patch(precision, n=1024, n_rho=256, rho_max=3.0, q_max=2)
    el = wl.element
    return dataclasses.replace(wl, element=dataclasses.replace(el, q=workloads.complex_normal((el.q.shape[0], 8), 81)))


@pytest.fixture(scope="module")
def eight_mbf_oracle():
    """The oracle table of the eight-MBF patch (FP64 definitions, the same for both GPU
    precisions), computed once for the module."""
    return cc.oracle_table(_eight_mbf_patch("fp64"))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_eight_mbfs_table_and_fill(torch_cuda, eight_mbf_oracle, precision):
    """The largest MBF count the ABI takes (M = 8: 64 pairs, four chunks of the
    integrand's pair loop, four series chunks per harmonic in the back-projection, the
    per-row fill): the whole table and a small array's fill against the oracle."""
    torch = torch_cuda
    wl = _eight_mbf_patch(precision)
    assert wl.element.n_mbf == 8
    ctx, got = cc.gpu_table(wl)
    ref, nodes, hq = eight_mbf_oracle
    err = cc.rel_err_per_pair(got, ref).max()
    pos = workloads.poisson_disc(5, 1.2, 0.5, seed=82)
    a, m = len(pos), 8
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    z = torch.zeros((a * m, a * m), dtype=dt, device="cuda:0")
    ctx.fill_reduced_matrix(torch.tensor(pos, device="cuda:0"), None, z)
    pairs = [(i, j) for i in range(a) for j in range(a)]
    blocks = cc.oracle_fill_entries(wl, hq, nodes, pos, np.zeros(a, dtype=np.int32), pairs)
    zref = np.zeros((a * m, a * m), dtype=np.complex128)
    for (i, j), blk in zip(pairs, blocks):
        zref[i * m:(i + 1) * m, j * m:(j + 1) * m] = blk
    ferr = np.abs(z.cpu().numpy() - zref).max() / np.abs(zref).max()
    print(precision, "M = 8: table rel err", err, "fill rel err", ferr, "fill form", ctx.info()["fill_form"])
    assert err < TOL[precision] and ferr < TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_residual_adjoint_matches_general_adjoint(torch_cuda, precision):
    """cfft_fill_backward_residual (dL/dZ' = 2 r v^H of L = sum |Z' v - t|^2, formed on the
    device from v and r) against cfft_fill_backward on the same matrix formed by PyTorch:
    position and substrate gradients, 4 rotation classes."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch(precision, n=1024, n_rho=512, rho_max=5.0, q_max=3, rotation_classes=4)
    ctx = cc.gpu_context(wl, options={cfft.OPT_DERIVATIVES: 1})
    prec = cfft.CFFT_FP64 if precision == "fp64" else cfft.CFFT_FP32_MIXED
    ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, prec, 4)
    pos = workloads.poisson_disc(60, 2.4, 0.4, seed=43)
    rot = workloads.rotations(len(pos), seed=43)
    a, m = len(pos), 4
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    v = torch.tensor(workloads.complex_normal(a * m, 62), device="cuda:0").to(dt)
    r = torch.tensor(workloads.complex_normal(a * m, 63), device="cuda:0").to(dt)
    g = (2 * r[:, None] * v.conj()[None, :]).contiguous()
    pos_t, rot_t = torch.tensor(pos, device="cuda:0"), torch.tensor(rot, device="cuda:0")
    ref_p, ref_t = ctx.fill_backward(pos_t, rot_t, g)
    gp, gt = ctx.fill_backward_residual(pos_t, rot_t, v, r)
    ep = ((gp - ref_p).abs().max() / ref_p.abs().max()).item()
    et = ((gt - ref_t).abs() / ref_t.abs()).max().item()
    print(precision, "residual form vs general adjoint: pos", ep, "eps/h", et)
    tol_p, tol_t = (1e-11, 1e-11) if precision == "fp64" else (2e-5, 5e-5)
    assert ep < tol_p and et < tol_t


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


def test_empty_inputs(torch_cuda):
    """Empty inputs: a fill of no elements and a batch of no items are refused as
    arguments (CFFT_ERR_ARG); spectra at no points are an empty result."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    wl = cc.small_patch("fp32", n=1024, n_rho=128, rho_max=3.0, q_max=1)
    ctx, _ = cc.gpu_table(wl)
    pos = torch.zeros((0, 2), dtype=torch.float64, device="cuda:0")
    z = torch.zeros((0, 0), dtype=torch.complex64, device="cuda:0")
    with pytest.raises(cfft.CfftError) as ei:
        ctx.fill_reduced_matrix(pos, None, z)
    assert ei.value.status == 1
    with pytest.raises(cfft.CfftError) as ei:
        ctx.tabulate_batch([], 1, 3.0, 128, cfft.CFFT_FP32_MIXED)
    assert ei.value.status == 1
    out = ctx.mbf_spectra(torch.zeros((0, 2), dtype=torch.complex64, device="cuda:0"))
    assert tuple(out.shape) == (0, 2, 4, 2)
