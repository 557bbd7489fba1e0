#!/usr/bin/env python
"""Benchmark of the C-FFT hot path on GB300.

Headline: C-FFT table samples/s on the rooftop-patch workload (200 rooftops,
M = 4 MBFs, all 16 MBF pairs, eps_r 4.4, h 0.03 lambda0, contour N = 16384,
|q| <= 16, 8192 rho points to 50 lambda0, FP32-mixed).  One step is one
cfft_tabulate_reactions call (contour + Green's function, MBF spectra and
harmonics, Taylor x pruned FFTs, back-projection) on inputs resident in HBM;
the L2 cache is flushed between timed steps.  Beside it, the same metric end
to end through the host-buffer C-ABI path, the plain FP64 GPU form of the same
tabulation, the reduced-matrix fill of the 10,000-element irregular array
(entries/s), the batched sweep, the differentiable fill, the roofline of the
dominant kernel, and the FP64 oracle timed on the host cores.  On a one-GPU run the
oracle leg also checks sampled outputs of each line against the FP64 oracle
(the FP32 and FP64 tables, the fill's element-pair blocks, one sweep item).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cfft|reference]
Under torchrun every rank runs its own replica of the workload (the path
shards into independent problems; no collective on the data path) and the
slowest rank's time sets the whole-job throughput.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}
N_SM = 152
FP32_LANES_PER_SM = 128


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


def fp32_peak_tflops(sm_mhz, n_sm=N_SM):
    """FP32 FMA pipe peak from unit counts: SMs x 128 lanes x 2 flops x clock (GB300: 152
    SMs; the bench passes the device's own count)."""
    return n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi sampling during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


TABLE_SIZE = {}


def table_workload():
    """The patch-m4 workload (sizes overridable for small profiling cases)."""
    return workloads.patch_m4(precision="fp32", **TABLE_SIZE)


FILL_SIZE = {}


def fill_workload():
    """Irregular array: 10,000 Poisson-disc elements (min spacing 0.5) in a disc of
    radius 60 lambda0, rotations in {0, 90}; table of the patch element to
    rho_max = 121 lambda0 with four rotation classes.  A smaller element count (for
    profiling) keeps the areal density: the disc radius scales with sqrt(A)."""
    wl = workloads.patch_m4(n=16384, n_rho=16384, rho_max=121.0, q_max=16, precision="fp32",
                            rotation_classes=4)
    a = FILL_SIZE.get("n_elements", 10000)
    pos, rot = workloads.irregular_array(n_elements=a, radius=60.0 * math.sqrt(a / 10000.0))
    return wl, pos, rot


def set_problem(ctx, wl):
    s = wl.substrate
    ctx.set_substrate(s.eps_r, s.h, s.k0)
    el = wl.element
    ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
    c = wl.contour
    ctx.build_contour(c.n, c.beta_max, c.beta_p, c.height, -1)


def table_samples(wl):
    m = wl.element.n_mbf
    classes = 3 if wl.rotation_classes == 4 else 1   # tabulated classes ((90,90) is derived)
    return classes * m * m * (2 * wl.q_max + 1) * wl.n_rho


def oracle_sample(wl, rows, workers, keep=False):
    """FP64 oracle on a bounded sample: harmonics at every contour node (needed by any
    rho), Bessel sums for the given rows, all pairs and harmonics.  keep: also return the
    contour nodes and the harmonics (for further exact evaluations on the same contour)."""
    from oracle import contour as oc, reaction as orx, spectra as osp
    el = wl.element
    bs = osp.BasisSet("rooftop", el.q, cx=el.cx, cy=el.cy, direction=el.direction,
                      half_len=el.half_len, width=el.width)
    c = wl.contour
    nodes = oc.contour_nodes(c.n, c.beta_max, c.beta_p, c.height)
    s = wl.substrate
    hq = orx.harmonics(bs, nodes["beta_c"], wl.qs, 128, s.eps_r, s.h, s.k0, workers=workers)
    z = orx.table_bessel(hq, wl.qs, nodes["beta_c"], nodes["weight"], wl.rho[rows])
    m = el.n_mbf
    z = z.reshape(m * m, len(wl.qs), len(rows))
    return (z, nodes, hq) if keep else z


def run_reference(args):
    """The oracle timed on the host cores (rank 0 only)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    wl = table_workload()
    workers = max(1, min(32, os.cpu_count() or 1))
    rows = np.linspace(0, wl.n_rho - 1, 8).astype(int)
    # warm-up: imports and the worker pool start (a small call)
    small = workloads.patch_m4(n=256, n_rho=16, rho_max=2.0, q_max=wl.q_max)
    for _ in range(args.warmup):
        oracle_sample(small, np.array([0, 5]), workers)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_sample(wl, rows, workers)
        times.append(time.perf_counter() - t0)
    samples = wl.element.n_mbf ** 2 * len(wl.qs) * len(rows)
    total = sum(times)
    value = samples * args.steps / total
    sample_desc = ("all %d contour nodes x 128 angles of harmonics, Bessel sums for %d of %d rho rows, "
                   "16 pairs x 33 harmonics" % (wl.contour.n, len(rows), wl.n_rho))
    line = {"impl": "reference", "metric": "C-FFT table samples/s", "value": value,
            "unit": "samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_desc(wl),
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": workers, "kind": "oracle",
                             "sample": sample_desc},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_desc(wl):
    return {"workload": "patch-m4: 200 rooftops, M=4 (16 pairs), eps_r=4.4, h=0.03 lambda0, "
                        "contour N=%d, |q|<=%d, %d rho points to %g lambda0, FP32-mixed"
                        % (wl.contour.n, wl.q_max, wl.n_rho, wl.rho_max),
            "table_samples_per_step": table_samples(wl), "l2": "flushed between timed steps",
            "parallelism": "replicas"}


def flush_l2(torch, buf):
    buf.zero_()


def bench_tabulation(torch, cfft, args, dev):
    wl = table_workload()
    ctx = cfft.Context(dev)
    set_problem(ctx, wl)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP32_MIXED, 1)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    infos = []
    clocks = ClockSampler(dev)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush_l2(torch, flush)
        evs[k][0].record(stream)
        ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP32_MIXED, 1)
        evs[k][1].record(stream)
        infos.append(ctx.info())
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    return wl, ctx, step_ms, infos, clk


def bench_fp64(torch, cfft, args, dev):
    """The plain FP64 GPU form of the same tabulation (FP64 arithmetic throughout, zero
    padding 8, 16-tap stencils, Taylor order for 1e-13), a few steps with the L2 flushed."""
    wl = table_workload()
    ctx = cfft.Context(dev)
    set_problem(ctx, wl)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP64, 1)   # warm-up
    stream = torch.cuda.current_stream(dev)
    steps = 2
    ms = []
    for _ in range(steps):
        flush_l2(torch, flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP64, 1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    inf = ctx.info()
    table = ctx.copy_table(host=True)      # after the timed steps: for the oracle comparison
    return {"metric": "C-FFT table samples/s (plain FP64 GPU form)",
            "value": table_samples(wl) * steps / (sum(ms) / 1e3), "unit": "samples/s",
            "ms_per_step": sum(ms) / steps, "steps": steps,
            "stages_ms": {k: inf["ms_" + k] for k in ("contour", "integrand", "fft", "backproject")},
            "info": {k: inf[k] for k in ("taylor_order", "sigma", "fft_len", "sub_len", "bp_taps",
                                         "bp_form", "spectra_tc")}, "_info": inf}, table


def fp64_roofline(inf, wl, fp64_peak):
    """Stages of the plain FP64 tabulation against the measured FP64 FMA peak: every flop
    of that form runs on the FP64 pipe (no tensor cores)."""
    fl = stage_flops(inf, wl)
    out = {}
    for k in ("contour", "integrand", "fft", "backproject"):
        t = inf["ms_" + k] / 1e3
        tf = fl[k]["algorithmic"] / t / 1e12
        out[k] = {"ms": inf["ms_" + k], "tflops": tf, "frac": tf / fp64_peak}
    return {"bound": "fp64", "peak_tflops": fp64_peak, "stages": out}


def bench_e2e(torch, cfft, args, dev, wl):
    """Same metric through the host-buffer C-ABI path: element arrays from host memory,
    table copied back to pinned host memory, inside the timed region."""
    ctx = cfft.Context(dev)
    el = wl.element
    centers = np.ascontiguousarray(np.stack([el.cx, el.cy], 1))
    h2d = centers.nbytes + el.direction.astype(np.int32).nbytes + el.half_len.nbytes + \
        el.width.nbytes + el.q.astype(np.complex128).nbytes
    out = None
    times = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = wl.substrate
        ctx.set_substrate(s.eps_r, s.h, s.k0)
        ctx.set_mbf_spectra(centers, el.direction, el.half_len, el.width, el.q)
        c = wl.contour
        ctx.build_contour(c.n, c.beta_max, c.beta_p, c.height, -1)
        ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP32_MIXED, 1)
        out = ctx.copy_table(out=out, host=True)
        t1 = time.perf_counter()
        if k >= args.warmup:
            times.append(t1 - t0)
    d2h = out.numel() * out.element_size()
    return {"value": table_samples(wl) * len(times) / sum(times), "unit": "samples/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}, out


def bench_fill(torch, cfft, args, dev):
    wl, pos, rot = fill_workload()
    ctx = cfft.Context(dev)
    set_problem(ctx, wl)
    if "block" in FILL_SIZE:
        ctx.set_option(cfft.OPT_FILL_BLOCK, FILL_SIZE["block"])
    t0 = time.perf_counter()
    ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP32_MIXED, 4)
    tab_s = time.perf_counter() - t0
    info = ctx.info()
    a, m = len(pos), wl.element.n_mbf
    z = torch.empty((a * m, a * m), dtype=torch.complex64, device=dev)
    dpos = torch.tensor(pos, dtype=torch.float64, device=dev)
    drot = torch.tensor(rot, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(1, min(args.warmup, 2))):
        ctx.fill_reduced_matrix(dpos, drot, z)
    steps = max(1, min(args.steps, 3))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        evs[k][0].record(stream)
        ctx.fill_reduced_matrix(dpos, drot, z)   # 12.8 GB output: far larger than L2
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = [x.elapsed_time(y) for x, y in evs]
    entries = float(a * m) ** 2
    res = {"metric": "Z-fill entries/s", "value": entries * steps / (sum(ms) / 1e3),
           "unit": "entries/s", "ms_per_step": sum(ms) / steps,
           "workload": "irregular array: A=%d Poisson-disc elements (min spacing 0.5) in a disc of "
                       "radius %.3g lambda0, rotations {0,90}, M=4, complex64 %dx%d, table to rho %g "
                       "lambda0 (%d points, 4 rotation classes)" % (a, 60.0 * math.sqrt(a / 10000.0), a * m,
                                                                   a * m, wl.rho_max, wl.n_rho),
           "table_ms": 1e3 * tab_s, "table_info": {k: info[k] for k in
                                                   ("taylor_order", "grid_half", "sigma", "fill_taps")}}
    # fill roofline: algorithmic FP32 work (interpolation + harmonic sum) vs the FP32 pipe,
    # and, in the tensor-core form, the TF32 products it executes (three per K step of the
    # per-cell GEMM: K = 2 n_harm padded to 8, N = 256, 128-pair tiles) vs the TF32 peak
    taps = info["fill_taps"]
    nh = 2 * wl.q_max + 1
    flops_per_pair = m * m * nh * (4 * taps + 8)
    sec = sum(ms) / steps / 1e3
    form = ctx.info()["fill_form"]
    res["form"] = {1: "per-row", 2: "bucketed, FP32 pipe", 3: "tensor cores"}.get(form, "none")
    res["algorithmic_tflops"] = flops_per_pair * float(a) ** 2 / sec / 1e12
    if form == 3:
        kpad = (2 * nh + 7) // 8 * 8
        res["tensor_tflops_executed"] = 3 * 2.0 * kpad * 256 * float(a) ** 2 / sec / 1e12
    res["hbm_gbs_write"] = entries * 8 / sec / 1e9
    fi = ctx.info()
    res["fill_table"] = {"err_est_on_tabulated_grid": fi["fill_err_est"], "refine": fi["fill_refine"],
                         "n_rho": fi["fill_n_rho"]}
    # element-pair blocks of every rotation class for the oracle comparison (after timing)
    pairs = fill_sample_pairs(pos, rot)
    blocks = [z[m * i:m * i + m, m * j:m * j + m].cpu().numpy().astype(np.complex128) for i, j in pairs]
    del z
    torch.cuda.empty_cache()
    return res, (wl, pos, rot, pairs, blocks)


FILL_BINS = ((0.4, 2.0), (20.0, 40.0), (60.0, 80.0), (100.0, 121.0))


def fill_sample_pairs(pos, rot, seed=91):
    """Element pairs (test m, basis n) of every rotation class (rot[m], rot[n]) in
    {0, 90 deg}^2, spread over the distances the fill's table covers: one diagonal block,
    then for each distance bin one pair of each class, measured from ten anchor basis
    elements of the class's basis rotation (bins the array does not reach are skipped)."""
    rot = np.asarray(rot)
    rng = np.random.default_rng(seed)
    pairs = [(int(np.flatnonzero(rot == 0)[0]),) * 2]
    for lo, hi in FILL_BINS:
        for cls in range(4):
            r_m, r_n = cls >> 1, cls & 1
            anchors = np.flatnonzero(rot == r_n)[:10]
            d = np.hypot(*(pos[:, None, :] - pos[None, anchors, :]).transpose(2, 0, 1))  # (A, anchors)
            cand = np.argwhere((d >= lo) & (d < hi) & (rot == r_m)[:, None])
            if len(cand) == 0:   # a smaller array (profiling runs) may not reach the bin
                continue
            k = rng.integers(len(cand))
            pairs.append((int(cand[k][0]), int(anchors[cand[k][1]])))
    return pairs


def class_harmonics(wl, nodes, cls, workers):
    """Oracle harmonics of rotation class cls on the table workload's contour nodes."""
    from oracle import reaction as orx, spectra as osp
    el = wl.element
    bs = osp.BasisSet("rooftop", el.q, cx=el.cx, cy=el.cy, direction=el.direction,
                      half_len=el.half_len, width=el.width)
    s = wl.substrate
    return orx.harmonics(bs, nodes["beta_c"], wl.qs, 128, s.eps_r, s.h, s.k0, *orx.rotation_angles(cls),
                         workers=workers)


def fill_parity(sample, table_wl, nodes, hq, workers=1):
    """The sampled blocks of the benchmarked fill against the oracle's exact fill (Bessel
    sums at each pair's exact rho) with the harmonics of the table workload's contour,
    which is the fill's own contour; max |err| over the blocks / max |oracle|.  hq holds
    the unrotated class; the other classes the pairs need are computed here."""
    from oracle import fill as ofill
    wl, pos, rot, pairs, blocks = sample
    same = (wl.contour == table_wl.contour and wl.q_max == table_wl.q_max and
            wl.substrate == table_wl.substrate)
    if not same:
        return {"skipped": "the fill's contour differs from the table workload's"}
    classes = sorted({2 * int(rot[i]) + int(rot[j]) for i, j in pairs})
    hq_by = {0: hq}
    for cls in classes:
        if cls not in hq_by:
            hq_by[cls] = class_harmonics(wl, nodes, cls, workers)
    ref = ofill.entries(hq_by, wl.qs, nodes["beta_c"], nodes["weight"], pos, rot, pairs)
    scale = max(np.abs(r).max() for r in ref)
    err = max(np.abs(g - r).max() for g, r in zip(blocks, ref)) / scale
    return {"max_rel_err_vs_oracle": float(err), "tolerance": 1e-5, "blocks": len(pairs),
            "rotation_classes": classes}


def bench_batch(torch, cfft, args, dev):
    """Batched sweep: 64 frequencies x 8 substrates, contours of 4k..64k samples, patch
    element (M = 4), |q| <= 16, 2048 rho points to 50 lambda0, FP32-mixed, one CUDA graph.
    Also returns the sampled rows of one item for the oracle comparison (sweep_sample)."""
    items = workloads.sweep_items()
    q_max, rho_max, n_rho = 16, 50.0, 2048
    el = table_workload().element
    ctx = cfft.Context(dev)
    ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
    out = torch.empty((len(items), 16, 2 * q_max + 1, n_rho), dtype=torch.complex64, device=dev)
    t0 = time.perf_counter()
    ctx.tabulate_batch(items, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, out=out, graph=True,
                       autotune=True)      # tunes, captures and runs the graph once
    first_s = time.perf_counter() - t0
    steps = max(1, min(args.steps, 2))
    times = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.tabulate_batch(items, q_max, rho_max, n_rho, cfft.CFFT_FP32_MIXED, out=out, graph=True)
        times.append(time.perf_counter() - t0)
    info = ctx.batch_info()
    samples = len(items) * 16 * (2 * q_max + 1) * n_rho
    ns = [it["n"] for it in items]
    res = {"metric": "C-FFT table samples/s (batched sweep)", "value": samples * steps / sum(times),
           "unit": "samples/s", "ms_per_sweep": 1e3 * sum(times) / steps,
           "ms_graph_replay": info["ms_graph"], "first_call_s": first_s,
           "workload": "64 frequencies (0.8..1.2) x 8 substrates (eps_r U[2,10], h U[0.02,0.1]); "
                       "contours n in [%d, %d] (mean %.0f); heights min(6 spacings, 3/rho_max); M=4; "
                       "|q|<=16; %d rho points to %g lambda0; FP32-mixed; one CUDA graph"
                       % (min(ns), max(ns), np.mean(ns), n_rho, rho_max),
           "first_wave_stage_ms": {k: info["ms_" + k] for k in ("integrand", "fft", "backproject")},
           "first_wave_note": "stage times of the first wave (of %d) from the tuning launches; the whole "
                              "sweep is ms_graph_replay" % info["waves"],
           "info": {k: v for k, v in info.items() if not k.startswith("ms_")}}
    return res, sweep_sample(out, items, q_max, rho_max, n_rho, el)


def sweep_sample(out, items, q_max, rho_max, n_rho, el):
    """The benchmarked sweep's item with the highest capped contour and the widest node
    spacing (the largest float32 growth exp(H rho)): its workload and three of its table
    rows (host copies, every pair and harmonic) for the comparison with the oracle."""
    x = np.array([it["height"] * rho_max for it in items])
    ns = np.array([it["n"] for it in items])
    bmax = np.array([it["beta_max"] for it in items])
    cand = np.flatnonzero(x >= x.max() - 1e-9)
    i = int(cand[np.argmax(bmax[cand] / ns[cand])])
    it = items[i]
    wl = workloads.TableWorkload("sweep-item", workloads.Substrate(it["eps_r"], it["h"], it["k0"]), el,
                                 workloads.ContourSpec(it["n"], it["beta_max"], it["beta_p"], it["height"]),
                                 q_max, rho_max, n_rho, "fp32")
    rows = np.array([0, n_rho // 2, n_rho - 1])
    got = np.asarray(out[i].cpu())[..., rows].astype(np.complex128)
    return {"item": i, "wl": wl, "rows": rows, "got": got, "height_times_rho_max": float(x[i])}


def sweep_parity(sample, workers):
    """The sampled sweep rows against the oracle: max over pairs of max |err| / max |oracle|."""
    t0 = time.perf_counter()
    ref = oracle_sample(sample["wl"], sample["rows"], workers)
    dt = time.perf_counter() - t0
    got = sample["got"]
    err = (np.abs(got - ref).reshape(ref.shape[0], -1).max(-1) /
           np.abs(ref).reshape(ref.shape[0], -1).max(-1))
    return {"max_rel_err_vs_oracle": float(err.max()), "tolerance": 1e-5, "item": sample["item"],
            "n": int(sample["wl"].contour.n), "height_times_rho_max": sample["height_times_rho_max"],
            "rows": sample["rows"].tolist(), "oracle_s": dt}


def bench_grad(torch, cfft, args, dev):
    """Differentiable fill: 2000 Poisson-disc elements in a disc of radius 25 lambda0, M = 4,
    L = sum |Z v - t|^2; forward (table + fill) and backward (table with substrate
    derivatives recomputed + adjoint fill), FP32-mixed."""
    from paper_1404_7357_gb300.autograd import FillProblem, ReducedMatrix
    wl = workloads.patch_m4(precision="fp32", rotation_classes=4)
    pos, rot = workloads.poisson_disc(2000, 25.0, 0.5, seed=5), workloads.rotations(2000, seed=5)
    prob = FillProblem(wl.element, wl.substrate.k0, wl.contour, wl.q_max, wl.rho_max, wl.n_rho,
                       "fp32", rot=torch.tensor(rot, device=dev), device=dev)
    m = wl.element.n_mbf
    v = torch.tensor(workloads.complex_normal(2000 * m, 5), device=dev).to(torch.complex64)
    t = torch.tensor(workloads.complex_normal(2000 * m, 6), device=dev).to(torch.complex64)
    pos_t = torch.tensor(pos, device=dev, requires_grad=True)
    eh = torch.tensor([wl.substrate.eps_r, wl.substrate.h], dtype=torch.float64, device=dev,
                      requires_grad=True)
    res = []
    for k in range(2):
        pos_t.grad = None
        eh.grad = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        z = ReducedMatrix.apply(pos_t, eh, prob)
        loss = ((z @ v - t).abs() ** 2).sum()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        res.append((t1 - t0, t2 - t1))
    fw, bw = res[-1]
    # the backward's two parts: the table with its substrate derivatives (recomputed), the adjoint fill
    eps_r, h = (float(x) for x in eh.detach().cpu())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prob.tabulate(eps_r, h, derivatives=True)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    g = torch.zeros((2000 * m, 2000 * m), dtype=torch.complex64, device=dev)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    prob.ctx.fill_backward(pos_t.detach(), prob.rot, g)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    return {"metric": "objective + gradient (2A + 2 parameters) per second", "value": 1.0 / (fw + bw),
            "unit": "gradients/s", "forward_ms": 1e3 * fw, "backward_ms": 1e3 * bw,
            "backward_table_ms": 1e3 * (t1 - t0), "backward_adjoint_fill_ms": 1e3 * (t3 - t2),
            "workload": "A=2000 Poisson-disc elements in a disc of radius 25 lambda0, rotations "
                        "{0,90}, M=4, table of patch-m4 (4 classes), FP32-mixed; L=sum|Zv-t|^2",
            "grad_norm_pos": float(pos_t.grad.norm()), "grad_eps_h": eh.grad.tolist()}


def bench_solve(torch, cfft, args, dev):
    """Reduced system of the 2,000-element array (M = 4: an 8,000 x 8,000 complex matrix, the
    gradient workload's layout): FP32 fill, delta-gap port excitation, then the LU solve in
    complex64, and FP32 factorization + FP64 refinement on a complex128 copy of the same
    matrix; times from the library's CUDA events (factorization, solve)."""
    wl = workloads.patch_m4(precision="fp32", rotation_classes=4)
    pos, rot = workloads.poisson_disc(2000, 25.0, 0.5, seed=5), workloads.rotations(2000, seed=5)
    ctx = cfft.Context(dev)
    set_problem(ctx, wl)
    ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, cfft.CFFT_FP32_MIXED, 4)
    m = wl.element.n_mbf
    n = 2000 * m
    z = torch.empty((n, n), dtype=torch.complex64, device=dev)
    ctx.fill_reduced_matrix(torch.tensor(pos, device=dev), torch.tensor(rot, dtype=torch.int32, device=dev), z)
    port = 37
    amps = torch.ones(2000, dtype=torch.complex64, device=dev)
    v = ctx.port_excitation(port, amps)
    res = {"workload": "A=2000 Poisson-disc elements in a disc of radius 25 lambda0, rotations {0,90}, M=4: "
                       "dense %d x %d reduced matrix, delta-gap port on basis function %d" % (n, n, port),
           "flops_per_factorization": 8.0 * n ** 3 / 3.0}
    for name, mat, refine in (("complex64", z, False), ("complex128_refined", None, True)):
        if mat is None:
            mat = z.to(torch.complex128)
            vv = v.to(torch.complex128)
        else:
            vv = v
        runs = []
        for _ in range(2):
            i_red = ctx.solve_reduced(mat, vv, refine=refine)
            runs.append(ctx.solve_info())
        inf = runs[-1]
        r = {"ms_factor": inf["ms_factor"], "ms_solve": inf["ms_solve"], "residual": inf["residual"],
             "refinements": inf["refinements"],
             "factor_tflops": res["flops_per_factorization"] / (inf["ms_factor"] / 1e3) / 1e12}
        if name == "complex64":
            ip = ctx.port_currents(port, i_red)
            r["port_current_mean_abs"] = float(ip.abs().mean())
        res[name] = r
        del mat
    del z
    torch.cuda.empty_cache()
    return res


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(torch, value):
    """The slowest rank's value (the whole job ends with it); CPU tensors under gloo."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([value], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return value


def whole_job_rate(units_per_rank_step, steps, world, max_seconds):
    """Units all ranks processed per second of the slowest rank: every rank runs its own
    replica of the workload (weak scaling), so the job does world x the units of one."""
    return units_per_rank_step * steps * world / max_seconds


def table_rel_err(table, ref, rows):
    """Max over MBF pairs of max |table - ref| / max |ref| on the sampled rows: `table` the
    (1, pairs, harmonics, n_rho) host copy of a one-class tabulation, `ref` the oracle's
    (pairs, harmonics, rows) sample."""
    got = np.asarray(table)[0][..., rows].astype(np.complex128)
    err = np.abs(got - ref).reshape(ref.shape[0], -1).max(-1) / np.abs(ref).reshape(ref.shape[0], -1).max(-1)
    return float(err.max())


def stage_flops(inf, wl):
    """Work of each tabulation stage for one launch, split by pipe: "fp32" = algorithmic
    flops on the FP32 pipe, "tensor" = the tensor-core flops the stage executed (three TF32
    products per term, as the library counts them), "algorithmic" = the stage's arithmetic
    counted once whichever pipe ran it.  The back-projection's matrix forms evaluate the
    quadrature as interpolation-matrix products (8 flops per complex MAC) plus the node
    stencils added into the matrices (weights + 2 taps + 16 flops each); "per_node_unit" is the
    gather form's (8 taps + 8) flops per (rho, alpha') node and series, the scope table's
    unit, which the matrix form beats by sharing each stencil across a chunk of series."""
    m = wl.element.n_mbf
    L = inf["sub_len"]
    taps = inf["bp_taps"]
    form = inf.get("bp_form", 0)
    per_node = inf["work_bp_nodes"] * (8.0 * taps + 8.0)
    if form in (1, 2, 3):
        prod = 8.0 * inf["work_bp_macs"]
        # a stencil: its weights (Lagrange: prefix and suffix products, 4 flops a tap; ES:
        # one Horner polynomial of degree taps + 1 per tap) plus 2 taps fused multiply-adds
        # into the A and B rows and 16 for its position and phase
        weights = 2.0 * taps * (taps + 1) if inf.get("bp_kernel", 0) == 1 else 4.0 * taps
        sten = (weights + 2.0 * taps + 16.0) * inf["work_bp_stencils"]
        bp = {"algorithmic": prod + sten, "fp32": sten if form == 3 else prod + sten,
              "tensor": inf.get("tc_flops_backproject", 0.0) if form == 3 else 0.0}
    else:
        bp = {"algorithmic": per_node, "fp32": per_node, "tensor": 0.0}
    bp["per_node_unit"] = per_node
    gemm = inf["work_points"] * 2 * 8.0 * inf["n_basis"] * m           # both MBF spectra (Eq. 11)
    rest = inf["work_points"] * m * m * (8.0 * inf["n_harm"] + 30.0)    # kernel + harmonic DFT
    tc_int = inf.get("tc_flops_integrand", 0.0) if inf.get("spectra_tc", 0) else 0.0
    fft = inf["work_subffts"] * 5.0 * L * math.log2(L)
    return {
        "contour": {"algorithmic": wl.contour.n * 200.0, "fp32": wl.contour.n * 200.0, "tensor": 0.0},
        "integrand": {"algorithmic": gemm + rest, "fp32": rest if tc_int else gemm + rest, "tensor": tc_int},
        "fft": {"algorithmic": fft, "fp32": fft, "tensor": 0.0},
        "backproject": bp,
    }


# DRAM bytes (read + write) per launch of each table kernel on the full patch-m4 workload,
# from one ncu capture of the current kernel (None: changed since its last capture);
# valid only for the default table sizes
KERNEL_DRAM_BYTES = {"integrand": 1.528e6 + 14.413e6, "fft": 88.564e6 + 8.654e6,
                     "backproject": 17.955e6 + 0.047e6}


def pipe_peaks(peaks):
    """TFLOP/s of the FP32 pipe and of the TF32 tensor cores the roofline divides by: the
    library's microbenchmarks when the bench measured them ("micro"), else the FP32 unit
    count x the maximum clock and the bf16 GEMM peak x the nominal TF32 / bf16 ratio."""
    micro = peaks.get("micro")
    if micro:
        return micro["fp32"], micro["tf32"], "measured: cfft_measure_peak microbenchmarks on this GPU"
    return (fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0), peaks.get("n_sm", N_SM)),
            peaks.get("bf16_tflops", 1900.0) * 1.1 / 2.25,
            "derived: FP32 unit count x max SM clock; bf16 GEMM peak x 1.1 / 2.25 for TF32")


def roofline(infos, wl, peaks, clk):
    """Dominant kernel of the tabulation step and its fraction of the bounding pipe.  A
    stage that runs on two pipes (FP32 and tensor cores) is bounded below by
    max(FP32 flops / FP32 peak, tensor flops / TF32 peak); its bound is the pipe with the
    larger share and "frac" is that pipe's achieved rate over its peak (= the two-pipe bound
    over the measured time)."""
    inf = infos[-1]
    ms = {k: float(np.mean([i["ms_" + k] for i in infos])) for k in
          ("contour", "integrand", "fft", "backproject")}
    dominant = max(ms, key=ms.get)
    p32, ptc, source = pipe_peaks(peaks)
    fl = stage_flops(inf, wl)
    traffic = KERNEL_DRAM_BYTES if not TABLE_SIZE else {}
    stages = {}
    for k in ms:
        t = ms[k] / 1e3
        f = fl[k]
        t32, ttc = f["fp32"] / (p32 * 1e12), f["tensor"] / (ptc * 1e12)
        bound = "tensor" if ttc > t32 else "alu"
        st = {"ms": ms[k], "bound": bound,
              "fp32_flops": f["fp32"], "fp32_tflops": f["fp32"] / t / 1e12, "fp32_frac": t32 / t,
              "tensor_flops_executed": f["tensor"], "tensor_tflops": f["tensor"] / t / 1e12,
              "tensor_frac": ttc / t, "frac": max(t32, ttc) / t,
              "algorithmic_tflops": f["algorithmic"] / t / 1e12, "dram_bytes": traffic.get(k)}
        if "per_node_unit" in f:
            st["per_node_unit_tflops"] = f["per_node_unit"] / t / 1e12
        stages[k] = st
    d = stages[dominant]
    if d["bound"] == "tensor":
        achieved, peak, kind = d["tensor_tflops"], ptc, "TF32 tensor cores (kind::tf32)"
    else:
        achieved, peak, kind = d["fp32_tflops"], p32, "FP32 FMA pipe"
    return {"kernel": dominant, "bound": "tensor" if d["bound"] == "tensor" else "alu",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic.get(dominant),
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "peak_note": "%s; peak source: %s" % (kind, source),
            "peaks_tflops": {"fp32": p32, "tf32": ptc}, "stages": stages,
            "algorithmic_flops_per_launch": fl[dominant]["algorithmic"],
            "spectra_on_tensor_cores": bool(inf.get("spectra_tc", 0)), "bp_form": inf.get("bp_form", 0),
            "note": "per stage: FP32-pipe flops and executed tensor-core flops (three TF32 products "
                    "per term) against the measured peak of each pipe; frac = the two-pipe lower "
                    "bound on the stage's time over its measured time"}


def measure_peaks(cfft, dev, reps=5):
    """The device's FP32, FP64, TF32-tensor and bf16-tensor peaks from the library's
    microbenchmarks (TFLOP/s, best of reps launches each), with the SM clock sampled."""
    clocks = ClockSampler(dev)
    clocks.start()
    out = {}
    for name, which in (("fp32", cfft.PEAK_FP32), ("fp64", cfft.PEAK_FP64), ("tf32", cfft.PEAK_TF32),
                        ("bf16", cfft.PEAK_BF16)):
        out[name] = cfft.measure_peak(dev, which, reps)[0]
    out["clocks"] = clocks.stop()
    return out


def run_cfft(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    from paper_1404_7357_gb300 import cfft
    peaks = load_peaks()
    peaks["n_sm"] = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks["micro"] = measure_peaks(cfft, dev)

    if args.only_fill:
        fill, _ = bench_fill(torch, cfft, args, dev)
        if rank == 0:
            print(json.dumps({"fill": fill}), flush=True)
        return
    wl, ctx, step_ms, infos, clk = bench_tabulation(torch, cfft, args, dev)
    total_s = max_over_ranks(torch, sum(step_ms) / 1e3)
    samples = table_samples(wl)
    value = whole_job_rate(samples, args.steps, world, total_s)
    e2e, host_table = bench_e2e(torch, cfft, args, dev, wl)
    fp64, fp64_table = (None, None) if args.skip_fp64 else bench_fp64(torch, cfft, args, dev)
    fill, fill_sample = (None, None) if args.skip_fill else bench_fill(torch, cfft, args, dev)
    batch, batch_sample = (None, None) if args.skip_batch else bench_batch(torch, cfft, args, dev)
    grad = None if args.skip_grad else bench_grad(torch, cfft, args, dev)
    solve = None if args.skip_solve else bench_solve(torch, cfft, args, dev)
    launches = int(sum(i["launches"] for i in infos))
    line = {"metric": "C-FFT table samples/s", "value": value, "unit": "samples/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_desc(wl),
            "roofline": roofline(infos, wl, peaks, clk), "clocks": clk,
            "gpu_launches": launches, "e2e": e2e, "info": infos[-1]}
    if fp64 is not None:
        inf64 = fp64.pop("_info")
        if peaks.get("micro"):
            fp64["roofline"] = fp64_roofline(inf64, wl, peaks["micro"]["fp64"])
        line["fp64_gpu"] = fp64
    if fill is not None:
        p32, ptc, _ = pipe_peaks(peaks)
        fill["algorithmic_frac_of_fp32_peak"] = fill["algorithmic_tflops"] / p32
        if "tensor_tflops_executed" in fill:
            fill["tensor_peak_tflops_tf32"] = ptc
            fill["tensor_frac"] = fill["tensor_tflops_executed"] / ptc
        fill["hbm_frac_write"] = fill["hbm_gbs_write"] / peaks.get("hbm_gbs", 6800.0)
        line["fill"] = fill
    if batch is not None:
        line["batch"] = batch
    if grad is not None:
        line["grad"] = grad
    if solve is not None:
        p32, _, _ = pipe_peaks(peaks)
        solve["complex64"]["factor_frac_of_fp32_peak"] = solve["complex64"]["factor_tflops"] / p32
        line["solve"] = solve
    line["peaks_source"] = peaks["_source"]
    if peaks.get("micro"):
        line["peaks_measured"] = {"fp32_tflops": peaks["micro"]["fp32"], "fp64_tflops": peaks["micro"]["fp64"],
                                  "tf32_tflops": peaks["micro"]["tf32"], "bf16_tflops": peaks["micro"]["bf16"],
                                  "bf16_tflops_cublas": peaks.get("bf16_tflops"),
                                  "clocks": peaks["micro"]["clocks"],
                                  "how": "cfft_measure_peak: FMA chains (FP32, FP64) and tcgen05.mma "
                                         "M128 N256 (kind::tf32, kind::f16 bf16), best of 5 launches"}
    if rank == 0 and world == 1 and not args.skip_cpu:
        workers = max(1, min(32, os.cpu_count() or 1))
        rows = np.linspace(0, wl.n_rho - 1, 8).astype(int)
        t0 = time.perf_counter()
        ref, nodes, hq = oracle_sample(wl, rows, workers, keep=True)
        dt = time.perf_counter() - t0
        ns = ref.size
        line["cpu_baseline"] = {"value": ns / dt, "unit": "samples/s", "cores": workers,
                                "kind": "oracle",
                                "sample": "all %d contour nodes (harmonics), %d of %d rho rows, all "
                                          "16 pairs x 33 harmonics; %.1f s" % (wl.contour.n, len(rows),
                                                                               wl.n_rho, dt)}
        line["parity"] = {"max_rel_err_vs_oracle": table_rel_err(host_table, ref, rows),
                          "rows": rows.tolist(), "tolerance": 1e-5}
        if batch_sample is not None:
            try:   # one benchmarked sweep item against the oracle on three rows
                line["batch"]["parity"] = sweep_parity(batch_sample, workers)
            except Exception as e:
                line["batch"]["parity"] = {"error": repr(e)[:300]}
        if fill_sample is not None:
            try:   # the fill's sampled blocks against the exact fill on the same harmonics
                line["fill"]["parity"] = fill_parity(fill_sample, wl, nodes, hq, workers)
            except Exception as e:
                line["fill"]["parity"] = {"error": repr(e)[:300]}
        if fp64_table is not None:
            # the plain FP64 GPU form against the same oracle sample
            line["fp64_gpu"]["parity"] = {"max_rel_err_vs_oracle": table_rel_err(fp64_table, ref, rows),
                                          "rows": rows.tolist(), "tolerance": 1e-10}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cfft", choices=["cfft", "reference"])
    ap.add_argument("--skip-fill", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--only-fill", action="store_true", help="time the fill alone")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-grad", action="store_true")
    ap.add_argument("--skip-solve", action="store_true", help="skip the reduced-system solve")
    ap.add_argument("--skip-fp64", action="store_true", help="skip the plain FP64 GPU form")
    ap.add_argument("--table-n", type=int, help="contour samples (small profiling case)")
    ap.add_argument("--table-nrho", type=int, help="rho points (small profiling case)")
    ap.add_argument("--table-rho", type=float, help="rho_max (small profiling case)")
    ap.add_argument("--fill-elements", type=int, help="array size of the fill (small profiling case)")
    ap.add_argument("--fill-block", type=int, help="test elements per row block of the fill")
    args = ap.parse_args()
    if args.fill_elements is not None:
        FILL_SIZE["n_elements"] = args.fill_elements
    if args.fill_block is not None:
        FILL_SIZE["block"] = args.fill_block
    for k, v in (("n", args.table_n), ("n_rho", args.table_nrho), ("rho_max", args.table_rho)):
        if v is not None:
            TABLE_SIZE[k] = v
    if args.warmup < 3 and args.impl == "cfft":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_cfft(args)


if __name__ == "__main__":
    main()
