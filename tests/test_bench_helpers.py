"""The arithmetic bench.py reports beside its timings, checked on CPU with made-up
stage times: the FP32 peak from unit counts and clock, the samples of one
tabulation, the algorithmic work of each stage, the roofline of the dominant
kernel, the whole-job rate of replicas, the sampled parity checks, and the
assembly of the JSON line around stand-ins for the GPU stages."""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import bench  # noqa: E402
import workloads  # noqa: E402


def _info(**kw):
    inf = {"ms_contour": 0.03, "ms_integrand": 1.25, "ms_fft": 1.51, "ms_backproject": 1.66,
           "sub_len": 16384, "bp_taps": 12, "bp_form": 3, "work_bp_macs": 4.8e9,
           "work_bp_stencils": 6.2e7, "work_bp_nodes": 1.0e9, "work_points": 16384 * 128.0,
           "n_basis": 200, "n_harm": 33, "work_subffts": 25344.0, "spectra_tc": 1}
    inf.update(kw)
    return inf


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2070 MHz
    assert bench.fp32_peak_tflops(2070.0) == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert bench.fp32_peak_tflops(2070.0) == pytest.approx(80.55, abs=0.01)


def test_table_samples_of_the_headline_workload():
    wl = workloads.patch_m4(precision="fp32")
    # 1 class x 16 MBF pairs x 33 harmonics x 8192 rho points
    assert bench.table_samples(wl) == 16 * 33 * 8192
    wl4 = workloads.patch_m4(precision="fp32", rotation_classes=4)
    assert bench.table_samples(wl4) == 3 * 16 * 33 * 8192    # (90, 90) is derived, not tabulated


def test_stage_flops_per_form():
    wl = workloads.patch_m4(precision="fp32")
    m = wl.element.n_mbf
    inf = _info(tc_flops_backproject=1.2e11, tc_flops_integrand=3.2e11)
    fl = bench.stage_flops(inf, wl)
    assert fl["fft"]["algorithmic"] == pytest.approx(25344 * 5 * 16384 * 14) == fl["fft"]["fp32"]
    assert fl["fft"]["tensor"] == 0.0
    gemm = 16384 * 128 * 2 * 8 * 200 * m
    rest = 16384 * 128 * m * m * (8 * 33 + 30)
    assert fl["integrand"]["algorithmic"] == pytest.approx(gemm + rest)
    # spectra on the tensor cores: the GEMM leaves the FP32 pipe, the executed products count there
    assert fl["integrand"]["fp32"] == pytest.approx(rest) and fl["integrand"]["tensor"] == 3.2e11
    assert bench.stage_flops(_info(spectra_tc=0), wl)["integrand"]["fp32"] == pytest.approx(gemm + rest)
    # matrix forms: 8 flops per complex MAC plus the node stencils added into the matrices
    prod, sten = 8 * 4.8e9, (6 * 12 + 16) * 6.2e7
    bp = fl["backproject"]
    assert bp["algorithmic"] == pytest.approx(prod + sten)
    assert bp["fp32"] == pytest.approx(sten) and bp["tensor"] == 1.2e11      # form 3: products on tensor cores
    for form in (1, 2):
        f = bench.stage_flops(_info(bp_form=form), wl)["backproject"]
        assert f["algorithmic"] == bp["algorithmic"] and f["fp32"] == pytest.approx(prod + sten)
        assert f["tensor"] == 0.0
    # the scope table's per-node unit, and the gather form that does exactly that work
    assert bp["per_node_unit"] == pytest.approx(1.0e9 * (8 * 12 + 8))
    g = bench.stage_flops(_info(bp_form=0), wl)["backproject"]
    assert g["algorithmic"] == g["fp32"] == g["per_node_unit"] == pytest.approx(1.0e9 * (8 * 12 + 8))


def test_roofline_of_the_dominant_kernel():
    wl = workloads.patch_m4(precision="fp32")
    infos = [_info(ms_backproject=1.60, tc_flops_backproject=1.2e11),
             _info(ms_backproject=1.72, tc_flops_backproject=1.2e11)]
    peaks = {"sm_max_mhz": 2070.0, "micro": {"fp32": 75.0, "tf32": 1000.0}}
    r = bench.roofline(infos, wl, peaks, None)
    assert r["kernel"] == "backproject"                      # 1.66 ms mean, the longest stage
    fl = bench.stage_flops(infos[-1], wl)["backproject"]
    t32, ttc = fl["fp32"] / 75e12, fl["tensor"] / 1000e12
    # products on the tensor cores take the larger share of the two-pipe bound
    assert ttc > t32 and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(fl["tensor"] / 1.66e-3 / 1e12)
    assert r["peak"] == 1000.0 and "measured" in r["peak_note"]
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"]) == pytest.approx(ttc / 1.66e-3)
    assert r["algorithmic_flops_per_launch"] == fl["algorithmic"]
    st = r["stages"]["backproject"]
    assert st["fp32_frac"] == pytest.approx(t32 / 1.66e-3) and st["frac"] == pytest.approx(ttc / 1.66e-3)
    # a stage on the FP32 pipe alone: bound "alu", frac = FP32 rate / FP32 peak
    fft = r["stages"]["fft"]
    assert fft["bound"] == "alu" and fft["frac"] == pytest.approx(fft["fp32_tflops"] / 75.0)
    # DRAM traffic of the default sizes from the committed capture; none for other sizes
    assert r["traffic"] == bench.KERNEL_DRAM_BYTES["backproject"]
    # without the microbenchmarks: the derived peaks, labelled as such
    r2 = bench.roofline(infos, wl, {"sm_max_mhz": 2070.0, "bf16_tflops": 1900.0}, None)
    assert r2["peaks_tflops"]["fp32"] == pytest.approx(bench.fp32_peak_tflops(2070.0))
    assert r2["peaks_tflops"]["tf32"] == pytest.approx(1900.0 * 1.1 / 2.25) and "derived" in r2["peak_note"]
    bench.TABLE_SIZE["n"] = 2048
    try:
        assert bench.roofline(infos, wl, peaks, None)["traffic"] is None
    finally:
        bench.TABLE_SIZE.clear()


def test_fp64_roofline_counts_every_flop_on_the_fp64_pipe():
    wl = workloads.patch_m4(precision="fp64")
    inf = _info(bp_form=1, spectra_tc=0, ms_integrand=75.0, ms_fft=137.0, ms_backproject=245.0)
    r = bench.fp64_roofline(inf, wl, 1.2)
    fl = bench.stage_flops(inf, wl)
    for k in ("integrand", "fft", "backproject"):
        tf = fl[k]["algorithmic"] / (inf["ms_" + k] / 1e3) / 1e12
        assert r["stages"][k]["tflops"] == pytest.approx(tf)
        assert r["stages"][k]["frac"] == pytest.approx(tf / 1.2)


def test_whole_job_rate_counts_every_replica():
    # 2 ranks x 4 steps x 100 units, the slowest rank took 2 s
    assert bench.whole_job_rate(100.0, 4, 2, 2.0) == pytest.approx(400.0)
    assert bench.whole_job_rate(100.0, 4, 1, 2.0) == pytest.approx(200.0)


def test_peaks_fallback_is_labelled(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    p = bench.load_peaks()
    assert p["_source"] == "fallback" and p["hbm_gbs"] == 6800.0 and p["bf16_tflops"] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6791.0, "bf16_tflops": 1908.7}')
    p = bench.load_peaks()
    assert p["_source"] == "measured" and p["hbm_gbs"] == 6791.0
    assert math.isclose(p["bf16_tflops"], 1908.7)


def test_sweep_parity_compares_the_benchmarked_rows(monkeypatch):
    """sweep_parity picks the capped item with the widest node spacing and compares the
    tables it was given on the rows it asked the oracle for (the oracle is replaced by a
    stand-in here; only the indexing and the error measure are checked)."""
    import torch
    items = workloads.sweep_items(n_freq=4, n_sub=2, seed=4)
    q_max, rho_max, n_rho = 1, 50.0, 64
    rng = np.random.default_rng(1)
    table = rng.standard_normal((len(items), 16, 2 * q_max + 1, n_rho)) + 0j
    seen = {}

    def fake_oracle(wl, rows, workers):
        seen["n"], seen["rows"] = wl.contour.n, list(rows)
        i = [k for k, it in enumerate(items) if it["n"] == wl.contour.n and
             it["beta_max"] == wl.contour.beta_max][0]
        ref = table[i][..., rows].copy()
        ref[3, 1, 2] += 1e-3 * np.abs(ref[3]).max()          # one planted difference
        return ref
    monkeypatch.setattr(bench, "oracle_sample", fake_oracle)
    out = torch.tensor(table.astype(np.complex64))
    sample = bench.sweep_sample(out, items, q_max, rho_max, n_rho, workloads.patch_rooftops())
    r = bench.sweep_parity(sample, 1)
    x = np.array([it["height"] * rho_max for it in items])
    spacing = np.array([it["beta_max"] / it["n"] for it in items])
    assert x[r["item"]] == pytest.approx(x.max())
    assert spacing[r["item"]] == max(spacing[x >= x.max() - 1e-9])
    assert seen["rows"] == [0, n_rho // 2, n_rho - 1] and seen["n"] == items[r["item"]]["n"]
    assert r["max_rel_err_vs_oracle"] == pytest.approx(1e-3, rel=1e-3)


def test_table_rel_err_per_pair_normalisation():
    """The bench's parity figure: per MBF pair, max |err| over harmonics and sampled rows
    over that pair's max |oracle|, then the worst pair (a torch host table or an array)."""
    import torch
    rng = np.random.default_rng(3)
    table = rng.standard_normal((1, 4, 3, 50)) + 1j * rng.standard_normal((1, 4, 3, 50))
    rows = np.array([0, 7, 49])
    ref = table[0][..., rows].copy()
    ref[1] *= 1e3                          # a large pair: its error counts relative to itself
    got = table.copy()
    got[0, 1][..., rows] = ref[1] * (1 + 1e-6)
    got[0, 2, 0, 7] += 1e-4 * np.abs(ref[2]).max()
    err = bench.table_rel_err(torch.tensor(got), ref, rows)
    assert err == pytest.approx(1e-4, rel=1e-6)
    assert bench.table_rel_err(got, ref, rows) == err


def test_fill_sample_pairs_cover_the_distance_bins():
    pos, rot = workloads.irregular_array()
    pairs = bench.fill_sample_pairs(pos, rot)
    assert len(pairs) == 17 and pairs[0][0] == pairs[0][1]
    d = [float(np.hypot(*(pos[i] - pos[j]))) for i, j in pairs]
    cls = [2 * int(rot[i]) + int(rot[j]) for i, j in pairs]
    for b, (lo, hi) in enumerate(bench.FILL_BINS):
        assert all(lo <= x < hi for x in d[1 + 4 * b:5 + 4 * b])
        assert cls[1 + 4 * b:5 + 4 * b] == [0, 1, 2, 3]               # every rotation class per bin
    assert bench.fill_sample_pairs(pos, rot) == pairs                 # seeded


def test_fill_parity_measure():
    """fill_parity compares the blocks it is given with the oracle's exact fill (tiny
    synthetic harmonics here) and refuses a fill whose contour is not the table's."""
    from oracle import contour as oc
    from oracle import fill as ofill
    wl = workloads.patch_m4(n=64, n_rho=32, rho_max=5.0, q_max=2)
    nodes = oc.contour_nodes(wl.contour.n, wl.contour.beta_max, wl.contour.beta_p, wl.contour.height)
    rng = np.random.default_rng(5)
    hq = rng.standard_normal((4, 4, 5, 64)) * 1e-3 + 1j * rng.standard_normal((4, 4, 5, 64)) * 1e-3
    pos = np.array([[0.0, 0.0], [1.0, 0.5], [-2.0, 1.0]])
    rot = np.zeros(3, dtype=np.int32)
    pairs = [(0, 0), (0, 1), (2, 1)]
    blocks = list(ofill.entries({0: hq}, wl.qs, nodes["beta_c"], nodes["weight"], pos, rot, pairs))
    assert bench.fill_parity((wl, pos, rot, pairs, blocks), wl, nodes, hq)["max_rel_err_vs_oracle"] == 0.0
    scale = max(np.abs(b).max() for b in blocks)
    blocks[2] = blocks[2].copy()
    blocks[2][1, 3] += 1e-4 * scale
    r = bench.fill_parity((wl, pos, rot, pairs, blocks), wl, nodes, hq)
    assert r["max_rel_err_vs_oracle"] == pytest.approx(1e-4, rel=1e-9) and r["blocks"] == 3
    other = workloads.patch_m4(n=128, n_rho=32, rho_max=5.0, q_max=2)
    assert "skipped" in bench.fill_parity((other, pos, rot, pairs, blocks), wl, nodes, hq)


def test_fill_parity_rotated_classes():
    """With rotated elements fill_parity computes the harmonics of each class the pairs
    need (only the unrotated class is handed in): exact blocks give zero error, a block
    computed with the unrotated class in place of a mixed one does not."""
    from oracle import contour as oc
    from oracle import fill as ofill
    wl = workloads.patch_m4(n=64, n_rho=32, rho_max=5.0, q_max=2)
    c = wl.contour
    nodes = oc.contour_nodes(c.n, c.beta_max, c.beta_p, c.height)
    hq = {cls: bench.class_harmonics(wl, nodes, cls, 1) for cls in range(4)}
    pos = np.array([[0.0, 0.0], [1.0, 0.5], [-2.0, 1.0]])
    rot = np.array([0, 1, 1], dtype=np.int32)
    pairs = [(0, 0), (0, 1), (1, 0), (2, 1)]            # classes 0, 1, 2, 3
    blocks = list(ofill.entries(hq, wl.qs, nodes["beta_c"], nodes["weight"], pos, rot, pairs))
    r = bench.fill_parity((wl, pos, rot, pairs, blocks), wl, nodes, hq[0])
    assert r["max_rel_err_vs_oracle"] == 0.0 and r["rotation_classes"] == [0, 1, 2, 3]
    wrong = ofill.entries({0: hq[0], 1: hq[0]}, wl.qs, nodes["beta_c"], nodes["weight"], pos, rot, [(0, 1)])
    expect = np.abs(wrong[0] - blocks[1]).max() / max(np.abs(x).max() for x in blocks)
    blocks[1] = wrong[0]
    got = bench.fill_parity((wl, pos, rot, pairs, blocks), wl, nodes, hq[0])["max_rel_err_vs_oracle"]
    assert expect > 1e-8 and got == pytest.approx(expect, rel=1e-12)


def test_bench_line_assembly_with_stand_in_stages(monkeypatch, capsys):
    """run_cfft's assembly of the JSON line, on CPU: the GPU stages are replaced by
    stand-ins that return what the real ones return (a small table workload, tables equal
    to the oracle's, fill blocks from the oracle's exact fill), while the oracle legs run
    for real.  Checks the keys the line must carry and that each parity entry is computed
    on the data it names."""
    import json
    import types
    import torch
    from oracle import fill as ofill
    from tests import cfft_cases as cc

    wl = workloads.patch_m4(n=64, n_rho=32, rho_max=2.0, q_max=2)
    ref_full, nodes, hq = cc.oracle_table(wl)
    table = ref_full.astype(np.complex64)                       # (1, 16, 5, 32)
    pos = np.array([[0.0, 0.0], [0.9, 0.4], [-1.0, 0.5]])
    rot = np.zeros(3, dtype=np.int32)
    pairs = [(0, 0), (1, 0), (2, 1)]
    blocks = list(ofill.entries({0: hq[0]}, wl.qs, nodes["beta_c"], nodes["weight"], pos, rot, pairs))
    infos = [dict(_info(), launches=6, n_basis=200, n_harm=5, sub_len=256) for _ in range(2)]

    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: types.SimpleNamespace(multi_processor_count=152))
    monkeypatch.setattr(bench, "measure_peaks", lambda *a: {"fp32": 75.0, "fp64": 1.2, "tf32": 1000.0,
                                                             "bf16": 1950.0, "clocks": {"sm_mhz": 2070.0}})
    monkeypatch.setattr(bench, "bench_tabulation",
                        lambda *a: (wl, None, [4.5, 4.4], infos, {"sm_mhz": 2070.0, "reasons": []}))
    monkeypatch.setattr(bench, "bench_e2e", lambda *a: ({"value": 1.0, "unit": "samples/s",
                                                         "h2d_bytes_per_step": 1, "d2h_bytes_per_step": 1},
                                                        torch.tensor(table)))
    monkeypatch.setattr(bench, "bench_fp64", lambda *a: ({"metric": "fp64", "_info": dict(infos[0], bp_form=1)},
                                                        torch.tensor(ref_full)))
    monkeypatch.setattr(bench, "bench_fill", lambda *a: ({"algorithmic_tflops": 1.0, "tensor_tflops_executed": 2.0,
                                                         "hbm_gbs_write": 500.0},
                                                        (wl, pos, rot, pairs, blocks)))
    monkeypatch.setattr(bench, "bench_batch", lambda *a: ({"metric": "batch"}, {
        "item": 0, "wl": wl, "rows": np.array([0, 16, 31]), "got": ref_full[0][..., [0, 16, 31]],
        "height_times_rho_max": 0.1}))
    monkeypatch.setattr(bench, "bench_grad", lambda *a: {"metric": "grad"})
    monkeypatch.setattr(bench, "bench_solve", lambda *a: {"complex64": {"factor_tflops": 7.5}})
    args = types.SimpleNamespace(steps=2, warmup=3, only_fill=False, skip_fp64=False, skip_fill=False,
                                 skip_batch=False, skip_grad=False, skip_cpu=False, skip_solve=False)
    bench.run_cfft(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "gpu_launches",
                "e2e", "cpu_baseline", "parity", "fp64_gpu", "fill", "batch", "grad"):
        assert key in line, key
    assert line["gpu_launches"] == 12 and line["steps"] == 2
    assert line["value"] == pytest.approx(bench.table_samples(wl) * 2 / 8.9e-3)
    assert line["parity"]["max_rel_err_vs_oracle"] < 1e-6              # complex64 copy of the oracle
    assert line["fp64_gpu"]["parity"]["max_rel_err_vs_oracle"] == 0.0   # the oracle itself
    assert line["fill"]["parity"]["max_rel_err_vs_oracle"] == 0.0
    assert line["batch"]["parity"]["max_rel_err_vs_oracle"] < 1e-10
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["roofline"]["bound"] in ("alu", "tensor") and 0 < line["roofline"]["frac"]
    assert line["peaks_measured"]["tf32_tflops"] == 1000.0 and "roofline" in line["fp64_gpu"]
    assert "_info" not in line["fp64_gpu"]
    assert line["solve"]["complex64"]["factor_frac_of_fp32_peak"] == pytest.approx(7.5 / 75.0)
