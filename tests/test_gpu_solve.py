"""The reduced system on the GPU (Section II): the reduced excitation V' = Q^H V (Eq. 4)
and delta-gap ports, the direct LU solution of Z' I' = V', and the port currents, all
through the C ABI.

- The LU solve against numpy's solve of the same matrix: orders that fill one panel,
  several panels and a ragged last panel; matrices that need row exchanges (zero
  diagonal, a permuted triangular matrix); FP32, FP64 and FP32 factorization with FP64
  refinement.  The bound is the precision's rounding times the condition number.
- A singular matrix is reported (CFFT_ERR_NUMERIC), not solved.
- End to end against the oracle: a 24-element patch array, the GPU fill, port
  excitation, solve and port currents against the oracle's exact fill, its reduced
  excitation, numpy's solve and its port currents; the difference is bounded by the
  fill's tolerance times the condition number of Z'.
"""
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


def _matrix(n, seed, kind="random"):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    if kind == "random":
        a += 3.0 * np.sqrt(n) * np.eye(n)            # well conditioned, no exchanges forced
    elif kind == "zero_diagonal":
        np.fill_diagonal(a, 0.0)                      # every step needs a row exchange
    elif kind == "permuted_triangular":
        u = np.triu(a) + 2.0 * np.sqrt(n) * np.eye(n)
        a = u[rng.permutation(n)]                     # pivots sit in scattered rows
    return a


def _solve(torch, cfft, a, b, dtype, refine=False, ld_pad=0):
    ctx = cfft.Context(0)
    n = a.shape[0]
    z = torch.zeros((n, n + ld_pad), dtype=dtype, device="cuda:0")
    z[:, :n] = torch.tensor(a, dtype=dtype)
    v = torch.tensor(b, dtype=dtype, device="cuda:0")
    x = ctx.solve_reduced(z, v, refine=refine)
    assert np.array_equal(z[:, :n].cpu().numpy(), a.astype(z.cpu().numpy().dtype))   # input untouched
    return x.cpu().numpy().astype(np.complex128), ctx.solve_info()


@pytest.mark.parametrize("n", [1, 64, 65, 300])
@pytest.mark.parametrize("kind", ["random", "zero_diagonal", "permuted_triangular"])
@pytest.mark.parametrize("mode", ["fp64", "fp32", "mixed"])
def test_lu_solve_against_numpy(torch_cuda, n, kind, mode):
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    if n == 1 and kind != "random":
        pytest.skip("one entry: nothing to exchange")
    a = _matrix(n, 7 + n, kind)
    b = np.random.default_rng(100 + n).standard_normal(n) + 1j * np.random.default_rng(200 + n).standard_normal(n)
    ref = np.linalg.solve(a, b)
    cond = np.linalg.cond(a)
    dtype = torch.complex64 if mode == "fp32" else torch.complex128
    x, info = _solve(torch, cfft, a, b, dtype, refine=(mode == "mixed"), ld_pad=3)
    err = np.abs(x - ref).max() / np.abs(ref).max()
    eps = 6e-8 if mode == "fp32" else 1.2e-16
    print(mode, kind, "n", n, "cond %.3g" % cond, "rel err %.3g" % err, "residual %.3g" % info["residual"],
          "refinements", info["refinements"])
    assert err < 50.0 * eps * cond * np.sqrt(n) + 1e-15
    # a small normwise backward error: |r| / |b| <= c eps (1 + |A| |x| / |b|)
    growth = 1.0 + np.linalg.norm(a, 2) * np.linalg.norm(ref) / np.linalg.norm(b)
    assert info["residual"] < 50.0 * eps * np.sqrt(n) * growth
    assert info["n"] == n and info["panel_width"] == 64


@pytest.mark.parametrize("n", [200, 1030])
def test_tensor_core_update_against_fp32_pipe(torch_cuda, n):
    """The complex64 trailing updates on the tensor cores (the complex product as a real
    GEMM, three TF32 products) against the same factorization with the updates on the FP32
    pipe and against numpy: several 128-row by 64-column tiles, a ragged last panel and
    ragged tiles (1030 = 16 x 64 + 6)."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    a = _matrix(n, 11 + n, "zero_diagonal")
    b = np.random.default_rng(5 + n).standard_normal(n) + 1j * np.random.default_rng(6 + n).standard_normal(n)
    ref = np.linalg.solve(a, b)
    cond = np.linalg.cond(a)
    xs, infos = {}, {}
    for simt in (0, 1):
        ctx = cfft.Context(0)
        ctx.set_option(cfft.OPT_SOLVE_SIMT, simt)
        z = torch.tensor(a, dtype=torch.complex64, device="cuda:0")
        v = torch.tensor(b, dtype=torch.complex64, device="cuda:0")
        xs[simt] = ctx.solve_reduced(z, v).cpu().numpy().astype(np.complex128)
        infos[simt] = ctx.solve_info()
    assert infos[0]["update_tc"] == 1 and infos[1]["update_tc"] == 0
    eps = 6e-8
    for simt in (0, 1):
        err = np.abs(xs[simt] - ref).max() / np.abs(ref).max()
        print("n", n, "simt", simt, "cond %.3g" % cond, "rel err %.3g" % err, "residual %.3g" % infos[simt]["residual"])
        assert err < 50.0 * eps * cond * np.sqrt(n)
    growth = 1.0 + np.linalg.norm(a, 2) * np.linalg.norm(ref) / np.linalg.norm(b)
    assert infos[0]["residual"] < 50.0 * eps * np.sqrt(n) * growth


@pytest.mark.parametrize("n,dtype", [(300, "complex64"), (1030, "complex128"), (2500, "complex128"),
                                     (4000, "complex64")])
def test_cluster_panel_against_grid_panel(torch_cuda, n, dtype):
    """The LU panel on one thread-block cluster (candidates and pivot rows read from the
    peers' shared memory, the cluster's hardware barrier) against the cooperative grid
    form (option SOLVE_GRID_PANEL): every row sees the same operations in the same order
    and every pivot is the same decision, so the two solutions are equal to the bit.  At
    2500 and 4000 the first panels are longer than the cluster form takes (2048 rows)
    and run on the grid, the others on the cluster."""
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    tdt = getattr(torch, dtype)
    a = _matrix(n, 31 + n, "zero_diagonal")
    b = np.random.default_rng(7 + n).standard_normal(n) + 1j * np.random.default_rng(8 + n).standard_normal(n)
    xs, infos = {}, {}
    for grid in (0, 1):
        ctx = cfft.Context(0)
        ctx.set_option(cfft.OPT_SOLVE_GRID_PANEL, grid)
        z = torch.tensor(a, dtype=tdt, device="cuda:0")
        v = torch.tensor(b, dtype=tdt, device="cuda:0")
        xs[grid] = ctx.solve_reduced(z, v).cpu().numpy()
        infos[grid] = ctx.solve_info()
        del z, v, ctx
    n_panels = (n + 63) // 64
    print("n", n, dtype, "cluster panels", infos[0]["cluster_panels"], "of", n_panels, "cluster",
          infos[0]["panel_cluster"], "ms factor cluster %.2f grid %.2f" % (infos[0]["ms_factor"],
                                                                          infos[1]["ms_factor"]))
    assert infos[1]["cluster_panels"] == 0 and infos[1]["panel_cluster"] == 0
    assert infos[0]["panel_cluster"] in (8, 16) and 0 < infos[0]["cluster_panels"] <= n_panels
    if n > 2048:
        assert infos[0]["cluster_panels"] < n_panels        # mixed: the first panels on the grid
    assert np.array_equal(xs[0], xs[1])


def test_singular_matrix_is_reported(torch_cuda):
    torch = torch_cuda
    from paper_1404_7357_gb300 import cfft
    n = 100
    a = _matrix(n, 3)
    a[:, 17] = 0.0                     # a zero column: no pivot for it
    with pytest.raises(cfft.CfftError) as ei:
        _solve(torch, cfft, a, np.ones(n), torch.complex128)
    assert ei.value.status == 5        # CFFT_ERR_NUMERIC


def test_reduced_excitation_and_ports_against_oracle(torch_cuda):
    """V' = Q^H V for a general V, the delta-gap form, and the port currents, against the
    oracle's definitions (Q in the caller's basis order)."""
    torch = torch_cuda
    from oracle import solve as osolve
    wl = cc.small_patch("fp64", n=1024, n_rho=256, rho_max=3.0, q_max=2)
    ctx = cc.gpu_context(wl)
    el = wl.element
    a_el, b_count = 7, el.q.shape[0]
    rng = np.random.default_rng(41)
    v = rng.standard_normal((a_el, b_count)) + 1j * rng.standard_normal((a_el, b_count))
    got = ctx.reduced_excitation(torch.tensor(v, device="cuda:0")).cpu().numpy()
    ref = osolve.reduced_excitation(el.q, v)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    port = 37
    amps = rng.standard_normal(a_el) + 1j * rng.standard_normal(a_el)
    got = ctx.port_excitation(port, torch.tensor(amps, device="cuda:0")).cpu().numpy()
    ref = osolve.port_excitation(el.q, port, amps)
    assert np.abs(got - ref).max() < 1e-14 * np.abs(ref).max()
    ired = rng.standard_normal(a_el * el.n_mbf) + 1j * rng.standard_normal(a_el * el.n_mbf)
    got = ctx.port_currents(port, torch.tensor(ired, device="cuda:0")).cpu().numpy()
    ref = osolve.port_currents(el.q, port, ired)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    from paper_1404_7357_gb300 import cfft
    with pytest.raises(cfft.CfftError):
        ctx.port_currents(b_count, torch.tensor(ired, device="cuda:0"))    # no such basis function


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_port_currents_end_to_end_against_oracle(torch_cuda, precision):
    """24-element patch array: GPU fill -> port excitation -> solve -> port currents, against
    the oracle's exact fill, excitation, numpy solve and port currents."""
    torch = torch_cuda
    from oracle import solve as osolve
    wl = cc.small_patch(precision, n=1024, n_rho=512, rho_max=5.0, q_max=3)
    ctx, _ = cc.gpu_table(wl)
    pos = workloads.poisson_disc(24, 2.4, 0.5, seed=21)
    a_el, m = len(pos), wl.element.n_mbf
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    z = torch.empty((a_el * m, a_el * m), dtype=dt, device="cuda:0")
    ctx.fill_reduced_matrix(torch.tensor(pos, device="cuda:0"), None, z)
    port = 37
    amps = np.exp(1j * np.linspace(0.0, 2.0, a_el))
    vred = ctx.port_excitation(port, torch.tensor(amps, dtype=dt, device="cuda:0"))
    ired = ctx.solve_reduced(z, vred, refine=False)
    ip = ctx.port_currents(port, ired).cpu().numpy().astype(np.complex128)
    # the same solve by numpy on the GPU's matrix: the solver alone
    zg = z.cpu().numpy().astype(np.complex128)
    ref_same = np.linalg.solve(zg, vred.cpu().numpy().astype(np.complex128))
    cond = np.linalg.cond(zg)
    eps = 6e-8 if precision == "fp32" else 1.2e-16
    err_solver = np.abs(ired.cpu().numpy() - ref_same).max() / np.abs(ref_same).max()
    # end to end: the oracle's exact fill and its reduced system
    nodes, hq = cc.oracle_harmonics(wl)
    pairs = [(i, j) for i in range(a_el) for j in range(a_el)]
    blocks = cc.oracle_fill_entries(wl, hq, nodes, pos, np.zeros(a_el, dtype=np.int32), pairs)
    zo = np.zeros((a_el * m, a_el * m), dtype=np.complex128)
    for (i, j), blk in zip(pairs, blocks):
        zo[i * m:(i + 1) * m, j * m:(j + 1) * m] = blk
    io = osolve.solve_reduced(zo, osolve.port_excitation(wl.element.q, port, amps))
    ipo = osolve.port_currents(wl.element.q, port, io)
    err_e2e = np.abs(ip - ipo).max() / np.abs(ipo).max()
    fill_tol = 1e-5 if precision == "fp32" else 1e-10
    print(precision, "cond(Z') %.3g" % cond, "solver vs numpy %.3g" % err_solver,
          "port currents vs oracle %.3g" % err_e2e, ctx.solve_info())
    assert err_solver < 50.0 * eps * cond * np.sqrt(a_el * m)
    assert err_e2e < 4.0 * cond * fill_tol
    if precision == "fp64":
        # FP32 factorization + FP64 refinement reaches the FP64 solution of the same matrix
        ir = ctx.solve_reduced(z, vred, refine=True).cpu().numpy()
        assert np.abs(ir - ref_same).max() < 50.0 * eps * cond * np.sqrt(a_el * m) * np.abs(ref_same).max()
        assert ctx.solve_info()["refinements"] >= 1
