#!/usr/bin/env python
"""Benchmark of the exact survey-field sampler (one JSON line on stdout).

A step is one pass of the whole hot path over one batch: circulant embedding
with its binary64 eigenvalues and positivity check, 64 realizations of
binary32 exact Gaussian fields with the fused lognormal + Poisson epilogue,
and the 64-bin power spectra of the 128 Gaussian fields and of the 128 count
maps with their mean and covariance (workload: 2D 512x512 survey in a
1024x1024 periodic grid, xi = 0.8/(1+(r/8)^2)^0.4, nbar = 2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 it runs under torch.distributed (one process per GPU); every rank
samples its own realization range (replicas, weak scaling) and rank 0 prints.
"--impl reference" times the CPU oracle on the same workload (bounded sample
per step) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "cauchy2d_n512_f32"
METRIC = "exact Gaussian/lognormal fields per sec (cells/s, % HBM roofline) vs plain FP64"
UNIT = "cells/s"


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-cufft-reference", action="store_true", help="skip the cuFFT reference timing")
    p.add_argument("--cpu-sample-realizations", type=int, default=8)
    p.add_argument("--serve-requests", type=int, default=10000)
    p.add_argument("--tune", action="store_true", help="autotune the sampler's chunk schedule before warm-up")
    p.add_argument("--mock-realizations", type=int, default=None,
                   help="mock_n128 workload: realizations per method (default 2000)")
    p.add_argument("--graph", action="store_true",
                   help="time replays of a captured plan (embedding computed once, per-realization path replayed)")
    p.add_argument("--lanes", type=int, default=2,
                   help="pipelines that alternate steps (own buffers and streams), so that one step's "
                        "sampler overlaps the previous step's spectra")
    p.add_argument("--embed-priority", default="high", choices=["high", "normal"],
                   help="priority of the embeddings' stream (high: the next step's embedding is not held up "
                        "behind the current step's sampler blocks)")
    p.add_argument("--embed-df", action="store_true",
                   help="eigenvalues through double-float transforms (CF_EMBED_DF) instead of binary64")
    p.add_argument("--fused", action="store_true",
                   help="square 2D grids: sampler and the fields' spectra through cf_sample_spectra")
    p.add_argument("--precision", default="all", choices=["all", "f64", "f32", "bf16_tc", "f16_tc"],
                   help="precision-sweep workload: run one precision only")
    return p.parse_args()


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------- roofline
SMS, LANES = 152, 128          # GB300: SMs, FP32 lanes per SM


def kernel_costs(wl, R, chunks):
    """Algorithmic bytes and operations per step of each kernel of the binary32
    path, 2D or 3D (FMA = 1 op).

    sample_rows: noise + last-axis transform of every embedded row; writes the
    pruned intermediate (R * prod(M[:-1]) * n[-1] complex64) and reads
    sqrt(lambda) once per launch; 76 ops of noise per embedded cell plus the
    row transforms.  icols (3D only): axis-1 pass between the intermediates.
    icols_fields_lp: last pass (axis 0), reads its intermediate, writes 2 fields
    + 2 count maps per realization; column transforms plus the Poisson step.
    pk_rows / pk_cols: fields in, half spectra out / in, for the Gaussian
    fields and the count maps."""
    import math
    n, m = list(wl.n), list(wl.m)
    d = len(n)
    F = 2 * R
    lg = lambda v: v.bit_length() - 1
    cells = math.prod(n)
    nbar = wl.nbar or 0.0
    inter1 = R * math.prod(m[:-1]) * n[-1] * 8
    costs = {"sample_rows_f32": {"bytes": inter1 + chunks * math.prod(m) * 4,
                                 "ops": R * math.prod(m) * 76 + R * math.prod(m[:-1]) * 4 * m[-1] * lg(m[-1])}}
    inter_last = R * m[0] * (cells // n[0]) * 8
    if d == 3:
        costs["icols_f32"] = {"bytes": inter1 + inter_last, "ops": R * m[0] * n[2] * 4 * m[1] * lg(m[1])}
    costs["icols_fields_lp_f32"] = {"bytes": inter_last + F * cells * 8,
                                    "ops": R * (cells // n[0]) * 4 * m[0] * lg(m[0])
                                    + F * cells * (30 + 10 + 4 * (nbar + 1))}
    half = F * (cells // n[-1]) * (n[-1] // 2 + 1) * 8
    costs["pk_rows_f32"] = {"bytes": 2 * (F * cells * 4 + half),
                            "ops": 2 * F * (cells // n[-1]) * 2 * n[-1] * lg(n[-1])}
    lines0 = F * (cells // (n[0] * n[-1])) * (n[-1] // 2 + 1)  # axis-0 lines of the half spectra
    costs["pk_cols_f32"] = {"bytes": 2 * half, "ops": 2 * lines0 * (4 * n[0] * lg(n[0]) + 8 * n[0])}
    return costs


def recorded_dominant():
    """The committed ncu record of the dominant kernel (largest share of the
    launch list), or {}."""
    try:
        with open(os.path.join(ROOT, "profiles", "dominant_kernel_traffic.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if
    it was taken on this workload and the current version of that kernel."""
    d = recorded_dominant()
    if d.get("kernel") == kernel and d.get("workload") == workload and d.get("current", False):
        return d["dram_bytes_per_launch"]
    return None


def step_bytes(wl, R):
    """The scope table's per-realization byte counts of the sampler path
    (steps b1-c2): floor = the outputs (2 fields, and 2 count maps when the
    lognormal + Poisson step runs) plus the amplitudes sqrt(lambda+) read
    once per batch of R; plan = floor plus the pruned intermediates written
    and read once (2D: M0 x n1 complex; 3D: M0 x M1 x n2 and M0 x n1 x n2)."""
    import numpy as np
    n, m = [int(v) for v in wl.n], [int(v) for v in wl.m]
    real = 4 if wl.dtype == "f32" else 8
    cells = int(np.prod(n))
    out = 2 * cells * (real + (4 if wl.nbar is not None and wl.dtype == "f32" else 0))
    amp = int(np.prod(m)) * real / R
    if len(n) == 1:
        inter = 0
    elif len(n) == 2:
        inter = m[0] * n[1]
    else:
        inter = m[0] * m[1] * n[2] + m[0] * n[1] * n[2]
    floor = out + amp
    return floor, floor + 2 * inter * 2 * real


def roofline(wl, R, timing, steps, hbm_peak, peak_kind, sm_mhz):
    per_kernel = {}
    for name, (launches, ms) in timing.items():
        base = name.split("<")[0]
        per_kernel.setdefault(base, [0, 0.0])
        per_kernel[base][0] += launches
        per_kernel[base][1] += ms
    launches_rows = per_kernel.get("sample_rows_f32", [steps, 0])[0]
    chunks = max(1, launches_rows // max(steps, 1))
    costs = kernel_costs(wl, R, chunks)
    # the kernel with the largest share of the ncu launch list (serialised
    # times; event times of kernels on concurrent streams overlap), else the
    # largest event time
    dom = recorded_dominant().get("kernel")
    if dom not in costs or per_kernel.get(dom, [0, 0.0])[1] <= 0:
        dom = max(per_kernel.items(), key=lambda kv: kv[1][1])[0]
    if dom not in costs:
        timed = [k for k in costs if per_kernel.get(k, [0, 0.0])[1] > 0]
        if not timed:
            return None, per_kernel  # no cost model for this path (binary64 workload)
        dom = max(timed, key=lambda k: per_kernel[k][1])
    launches, ms = per_kernel[dom]
    avg_s = ms / launches * 1e-3
    ops = costs[dom]["ops"] * steps / launches
    byts = costs[dom]["bytes"] * steps / launches
    clock = sm_mhz or 2070.0
    alu_peak = SMS * LANES * clock * 1e6 / 1e12
    achieved = ops / avg_s / 1e12
    hbm = byts / avg_s / 1e9
    # the measure of the sampler's scope table: algorithmic HBM bytes of the
    # dominant kernel per launch over its launch time, against the measured
    # copy bandwidth; the ALU view (algorithmic operations against the FP32
    # lane rate) is kept beside it, since these kernels are issue-bound
    return {"bound": "hbm", "kernel": dom, "achieved": round(hbm, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(hbm / hbm_peak, 4), "traffic": recorded_traffic(dom, wl.name),
            "peak_source": "%s copy bandwidth (MEASURED_PEAKS hbm_gbs)" % peak_kind
                           if peak_kind == "measured" else "fallback 6.8 TB/s",
            "bytes_per_launch": int(byts), "avg_launch_ms": round(avg_s * 1e3, 5), "launches": launches,
            "alu": {"achieved": round(achieved, 3), "peak": round(alu_peak, 2), "unit": "TOP/s",
                    "frac": round(achieved / alu_peak, 4), "ops_per_launch": int(ops),
                    "peak_source": "152 SMs x 128 FP32 lanes x %s SM clock %.0f MHz (one op per lane per cycle)"
                                   % ("sampled" if sm_mhz else "maximum", clock)}}, per_kernel


# --------------------------------------------------------------------- CPU oracle
def oracle_sample_run(wl, realizations, r0):
    """The oracle as it stands on a bounded sample of the workload: embed,
    `realizations` realizations (binary32 noise spec, binary64 arithmetic),
    lognormal + Poisson, power spectra of fields and count maps, mean/cov."""
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    e = oracle.embed(list(wl.n), wl.xi_kind, wl.amp, wl.scale, wl.beta, clamp=wl.clamp)
    fields = oracle.sample(wl.n, e["sqrt_lambda"], wl.seed, r0, realizations, 1 if wl.dtype == "f32" else 0)
    F = 2 * realizations
    G = fields.reshape(F, -1)
    cells = F * wl.cells_per_field
    if wl.nbar is not None:
        _, counts, _ = oracle.lognormal_poisson(G, wl.sigma2, wl.nbar, seed=wl.seed + 1000, field0=2 * r0)
    if wl.nbins:
        edges = oracle.bin_edges(oracle.BINS_LINEAR, wl.nbins, 0.0, wl.n[0] / 2)
        pk, _ = oracle.power_spectrum(fields.reshape((F,) + tuple(wl.n)), wl.n, edges)
        oracle.mean_cov(pk)
        if wl.nbar is not None:
            dg = oracle.counts_to_delta(counts, None)
            pkg, _ = oracle.power_spectrum(dg.reshape((F,) + tuple(wl.n)), wl.n, edges)
            oracle.mean_cov(pkg)
    dt = time.perf_counter() - t0
    return cells, dt, np


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(wl, realizations):
    import oracle
    oracle.build()
    cells, dt, _ = oracle_sample_run(wl, realizations, 0)
    return {"value": cells / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": "%d realization(s) (%d fields of %s) incl. embedding, lognormal+Poisson and spectra, "
                      "single-threaded C oracle, %.1f s" % (realizations, 2 * realizations,
                                                             "x".join(map(str, wl.n)), dt)}


def _oracle_worker(task):
    """One host process of the all-cores baseline: the oracle on `realizations`
    realizations starting at r0 (its own embedding included)."""
    name, realizations, r0 = task
    from paper_1406_6072_gb300 import workloads as W
    cells, dt, _ = oracle_sample_run(W.CONFIGS[name], realizations, r0)
    return cells


def cpu_baseline_all_cores(wl, per_core):
    """The same oracle run on every host core at once, parallel over
    realizations (one process per core, started with spawn), wall time."""
    import multiprocessing as mp

    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    tasks = [(wl.name, per_core, c * per_core) for c in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_worker, [(wl.name, 1, 10 ** 6 + c) for c in range(cores)])  # start-up outside the clock
        t0 = time.perf_counter()
        cells = sum(pool.map(_oracle_worker, tasks))
        dt = time.perf_counter() - t0
    return {"value": cells / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": "%d processes x %d realization(s) of %s, each with its own embedding, wall %.1f s"
                      % (cores, per_core, wl.name, dt)}


def run_reference(args):
    from paper_1406_6072_gb300 import workloads as W
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = W.CONFIGS[args.workload]
    import oracle
    oracle.build()
    R = max(1, args.cpu_sample_realizations // 2)
    if args.warmup > 0:
        oracle_sample_run(wl, R, 0)  # loads the library and touches the code paths once
    total_cells, total_t = 0, 0.0
    # each step is a bounded sample (one realization with its embedding); at
    # most 60 are timed so that the run ends within a few minutes
    steps = min(args.steps, 60)
    for k in range(steps):
        cells, dt, _ = oracle_sample_run(wl, R, (k + 1) * R)
        total_cells += cells
        total_t += dt
    value = total_cells / total_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "text": wl.text,
                                            "sample_realizations_per_step": R},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
                             "sample": "%d realization(s) per step of %s" % (R, wl.name)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------- precision sweep
def run_sweep(args):
    """Precision sweep: the 2D 2048^2 survey in 4096^2 (32 realizations per
    step) or the 3D 256^3 survey in 512^3 (4 per step), sampler + power
    spectrum in binary64, binary32 and the bf16 / fp16 tensor-core modes, the
    same seeds for all.  Reports cells/s per precision (embedding cached, as
    in a sweep over precisions of one spectrum); the error of each precision
    against the binary64 oracle is measured by tests/test_gpu_tc.py."""
    import torch

    from paper_1406_6072_gb300 import cf
    from paper_1406_6072_gb300 import workloads as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wl = W.CONFIGS[args.workload]
    stream = torch.cuda.Stream(dev)
    grid = cf.make_grid(wl.n)
    R, F = wl.R, 2 * wl.R
    bins = cf.make_bins(wl.nbins)
    out = {}
    clocks = ClockSampler(0)
    clocks.start()
    with torch.cuda.stream(stream):
        emb = cf.cf_embed(grid, cf.make_xi(wl.xi_kind, wl.amp, wl.scale, wl.beta), cf.CF_EMBED_CLAMP, stream)
        for name, dt in (("f64", cf.CF_F64), ("f32", cf.CF_F32), ("bf16_tc", cf.CF_BF16_TC),
                         ("f16_tc", cf.CF_F16_TC)):
            if args.precision not in ("all", name):
                continue
            fdt = cf.CF_F64 if dt == cf.CF_F64 else cf.CF_F32
            tdt = torch.float64 if fdt == cf.CF_F64 else torch.float32
            wsb = cf.cf_sample_workspace_size(emb, R, dt)
            ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=dev)
            fields = torch.empty((R, 2) + tuple(wl.n), dtype=tdt, device=dev)
            pkb = cf.cf_power_spectrum_workspace_size(grid, F, bins, fdt)
            pkws = torch.empty(pkb, dtype=torch.uint8, device=dev)
            pk = torch.empty((F, wl.nbins), dtype=torch.float64, device=dev)
            nm = torch.empty(wl.nbins, dtype=torch.int64, device=dev)
            mean = torch.empty(wl.nbins, dtype=torch.float64, device=dev)
            cov = torch.empty((wl.nbins, wl.nbins), dtype=torch.float64, device=dev)

            def step(k):
                cf.cf_sample(emb, wl.seed, k * R, R, dt, fields, ws, wsb, stream)
                cf.cf_power_spectrum(fields, fdt, grid, F, bins, pk, nm, mean, cov, pkws, pkb, stream)

            steps = max(3, min(args.steps, 20))
            for k in range(max(3, args.warmup)):
                step(k)
            torch.cuda.synchronize()
            cf.cf_kernel_timing(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(steps):
                step(100 + k)
            e1.record(stream)
            torch.cuda.synchronize()
            timing = cf.cf_kernel_timing_read()
            cf.cf_kernel_timing(0)
            ms = e0.elapsed_time(e1) / steps
            if dt in (cf.CF_BF16_TC, cf.CF_F16_TC):
                assert cf.cf_tc_faults(stream) == 0
            kern = {k: list(v) for k, v in timing.items()}
            out[name] = {"ms_per_step": ms, "cells_per_s": 2 * R * wl.cells_per_field / (ms * 1e-3),
                         "realizations_per_s": R / (ms * 1e-3),
                         "kernels_ms_per_step": {k: v[1] / steps for k, v in sorted(kern.items())}}
            del ws, fields, pkws
        emb.close()
    clk = clocks.stop()
    head = "f32" if "f32" in out else next(iter(out))
    side = "x".join(str(v) for v in wl.n)
    line = {"metric": f"cells/s per precision, {wl.ndim}D {side} sampler + power spectrum",
            "value": out[head]["cells_per_s"],
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "sweep", "data": "synthetic",
            "config": {"workload": wl.name, "text": wl.text, "realizations_per_step": R,
                       "note": "embedding cached across steps; errors vs the binary64 oracle: tests/test_gpu_tc.py"},
            "precisions": out, "clocks": clk}
    print(json.dumps(line))


# ---------------------------------------------------------------- section 3.3 / 3.4 experiment
def run_mock(args):
    """Synthetic analogue of the paper's CFHTLS analysis on a 128^2 map
    (workload mock_n128): cumulative information I(<= l) of the lognormal map
    rho = 1 + delta from the exact circulant embedding and from k-space
    sampling in periodic boxes of 1, 2 and 4 times the map (DC mode zeroed),
    section 3.3; and, for the exact sampler with the survey mask, the
    counts-in-cells histogram against the Poisson-lognormal prediction and the
    spectra of delta_g and of A* (section 3.4).  All steps are library calls."""
    import numpy as np
    import torch

    from paper_1406_6072_gb300 import cf
    from paper_1406_6072_gb300 import workloads as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wl = W.CONFIGS["mock_n128"]
    n = tuple(wl.n)
    cells = wl.cells_per_field
    Rtot = wl.R if args.mock_realizations is None else args.mock_realizations
    chunk = min(250, Rtot)
    Rtot = -(-Rtot // chunk) * chunk  # whole chunks
    nb = wl.nbins
    bins = cf.make_bins(nb, cf.CF_BINS_LOG, 1.0, n[0] / 2)
    grid = cf.make_grid(n)
    xi = cf.make_xi(wl.xi_kind, wl.amp, wl.scale, wl.beta)
    flags = cf.CF_EMBED_CLAMP | cf.CF_EMBED_LOG1P
    mask = torch.from_numpy(W.survey_mask(n, seed=wl.seed + 7)).to(dev)
    s = torch.cuda.Stream(dev)
    out = {"workload": wl.name, "text": wl.text, "realizations": Rtot}

    def spectra_of(emb, big_n, masked):
        F = 2 * Rtot
        pk_all = torch.empty((F, nb), dtype=torch.float64, device=dev)
        pkg_all = torch.empty_like(pk_all) if masked else None
        ast_all = torch.empty_like(pk_all) if masked else None
        hist_all = torch.empty((F, 42), dtype=torch.float64, device=dev) if masked else None
        wsb = cf.cf_sample_workspace_size(emb, chunk, cf.CF_F32)
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=dev)
        fields = torch.empty((chunk, 2) + big_n, dtype=torch.float32, device=dev)
        delta = torch.empty_like(fields)
        counts = torch.empty((chunk, 2) + big_n, dtype=torch.int32, device=dev)
        dcorner = torch.empty((chunk, 2) + n, dtype=torch.float32, device=dev)
        astar = torch.empty((chunk, 2) + n, dtype=torch.float32, device=dev)
        pkb = cf.cf_power_spectrum_workspace_size(grid, 2 * chunk, bins, cf.CF_F32)
        pkws = torch.empty(pkb, dtype=torch.uint8, device=dev)
        nm = torch.empty(nb, dtype=torch.int64, device=dev)
        for c0 in range(0, Rtot, chunk):
            lp = cf.make_lp(wl.sigma2, wl.nbar, counts, wl.seed + 1000, f=mask if masked else None, delta_out=delta)
            cf.cf_sample_lp(emb, wl.seed, c0, chunk, cf.CF_F32, fields, lp, ws, wsb, s)
            d = delta
            if big_n != n:
                cf.cf_copy_corner(delta, cf.CF_F32, cf.make_grid(big_n), grid, 2 * chunk, dcorner, s)
                d = dcorner
            sl = slice(2 * c0, 2 * c0 + 2 * chunk)
            cf.cf_power_spectrum(d, cf.CF_F32, grid, 2 * chunk, bins, pk_all[sl], nm, None, None, pkws, pkb, s)
            if masked:
                cf.cf_power_spectrum_counts(counts, mask, grid, 2 * chunk, bins, pkg_all[sl], nm, None, None, pkws,
                                            pkb, s)
                cf.cf_astar(counts, mask, cells, 2 * chunk, wl.nbar, wl.sigma2, astar, s)
                cf.cf_power_spectrum(astar, cf.CF_F32, grid, 2 * chunk, bins, ast_all[sl], nm, None, None, pkws,
                                     pkb, s)
                cf.cf_cic_histogram(counts, cells, 2 * chunk, mask, 42, hist_all[sl], None, None, s)
        return pk_all, pkg_all, ast_all, hist_all

    def info(pk_all):
        F = pk_all.shape[0]
        mean = torch.empty(nb, dtype=torch.float64, device=dev)
        cov = torch.empty((nb, nb), dtype=torch.float64, device=dev)
        cf.cf_mean_cov(pk_all, F, nb, mean, cov, s)
        I = torch.empty(nb, dtype=torch.float64, device=dev)
        wsb = cf.cumulative_information_workspace_size(nb)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        cf.cf_cumulative_information(mean, cov, nb, I, ws, wsb, s)
        torch.cuda.synchronize()
        return mean.cpu().numpy(), I.cpu().numpy()

    t0 = time.perf_counter()
    methods = {}
    with torch.cuda.stream(s):
        emb = cf.cf_embed(grid, xi, flags, s)
        pk, pkg, pka, hist = spectra_of(emb, n, False)
        mean, I = info(pk)
        methods["circulant"] = {"I": I.tolist(), "pk_mean": mean.tolist(), "embed_report": emb.report}
        emb.close()
        for bf in (1, 2, 4):
            emb = cf.cf_embed_periodic(grid, xi, bf, 2, 4, flags, s)
            big_n = tuple(2 * v for v in n) if bf == 4 else n
            pk, _, _, _ = spectra_of(emb, big_n, False)
            mean, I = info(pk)
            methods["box%d" % bf] = {"I": I.tolist(), "pk_mean": mean.tolist()}
            emb.close()
        # section 3.4 with the mask: counts in cells, delta_g and A* spectra
        emb = cf.cf_embed(grid, xi, flags, s)
        pk, pkg, pka, hist = spectra_of(emb, n, True)
        hm = torch.empty(42, dtype=torch.float64, device=dev)
        hc = torch.empty((42, 42), dtype=torch.float64, device=dev)
        cf.cf_mean_cov(hist, hist.shape[0], 42, hm, hc, s)
        pred = torch.empty(42, dtype=torch.float64, device=dev)
        cf.cf_cic_prediction(wl.sigma2, wl.nbar, mask, cells, 42, pred, s)
        mg, Ig = info(pkg)
        ma, Ia = info(pka)
        torch.cuda.synchronize()
        emb.close()
    hm, pred, hvar = hm.cpu().numpy(), pred.cpu().numpy(), torch.diagonal(hc).cpu().numpy()
    F = hist.shape[0]
    z = (hm - pred) / np.sqrt(np.maximum(hvar, 1e-12) / F)  # empirical per-bin scatter over the maps
    out["cumulative_information"] = methods
    out["counts_in_cells"] = {"mean_histogram": hm.tolist(), "prediction": pred.tolist(),
                              "max_abs_z": float(np.max(np.abs(z))), "fields": F}
    out["delta_g"] = {"pk_mean": mg.tolist(), "I": Ig.tolist()}
    out["astar"] = {"pk_mean": ma.tolist(), "I": Ia.tolist()}
    out["seconds"] = time.perf_counter() - t0
    print(json.dumps(out))


# ---------------------------------------------------------------- cuFFT reference
def cufft_reference(wl, R, stream, steps=10):
    """Context only: the inverse transforms of the same embedded grids by
    cuFFT (torch.fft, complex64, all R realizations in one batched call) plus
    the crop to the survey, inputs resident; no noise draw, no scaling, no
    lognormal/Poisson step, no spectra."""
    import torch
    if wl.dtype != "f32":
        return None
    m = tuple(wl.m)
    n = tuple(wl.n)
    x = torch.randn((R,) + m, dtype=torch.complex64, device=stream.device)
    crop = tuple(slice(0, v) for v in n)
    with torch.cuda.stream(stream):
        for _ in range(3):
            y = torch.fft.ifftn(x, dim=tuple(range(1, len(m) + 1)))[(slice(None),) + crop].contiguous()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            y = torch.fft.ifftn(x, dim=tuple(range(1, len(m) + 1)))[(slice(None),) + crop].contiguous()
        e1.record(stream)
        torch.cuda.synchronize()
    del x, y
    return {"ms_per_step": e0.elapsed_time(e1) / steps,
            "what": "cuFFT (torch.fft.ifftn) of the %d embedded %s complex64 grids + crop to %s; transforms only"
                    % (R, "x".join(map(str, m)), "x".join(map(str, n)))}


# --------------------------------------------------------------------- padding
def run_padding(args):
    """The 2D 512^2 workload's non-PSD generalised Cauchy spectrum embedded on
    2, 4 and 8 times the survey side: the clamping report (negative mass,
    realised-covariance error) against the cost of a whole step (embedding,
    sampler with lognormal + Poisson, both power spectra)."""
    import dataclasses

    import torch

    from paper_1406_6072_gb300 import cf
    from paper_1406_6072_gb300 import workloads as W
    from paper_1406_6072_gb300.pipeline import FieldPipeline
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = W.CONFIGS["cauchy2d_n512_padding"]
    stream = torch.cuda.Stream(dev)
    out = {}
    clocks = ClockSampler(0)
    clocks.start()
    for p in (2, 4, 8):
        wl = dataclasses.replace(base, factor=p)
        with torch.cuda.stream(stream):
            pipe = FieldPipeline(wl, dev, stream=stream)
            rep = pipe.embed()
            steps = max(3, min(args.steps, 30))
            for k in range(max(3, args.warmup)):
                pipe.step(r0=k * wl.R)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(steps):
                pipe.step(r0=(100 + k) * wl.R)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            pipe.close()
        out[f"factor_{p}"] = {"embedded_side": p * wl.n[0], "ms_per_step": ms,
                              "cells_per_s": pipe.cells_per_step / (ms * 1e-3),
                              "cov_error": rep["cov_error"], "neg_mass": rep["neg_mass"],
                              "lambda_min_over_max": rep["lambda_min"] / rep["lambda_max"],
                              "n_negative": rep["n_negative"]}
        del pipe
    clk = clocks.stop()
    line = {"metric": "clamping error and cells/s per embedding factor, 2D 512^2 step", "unit": UNIT,
            "value": out["factor_2"]["cells_per_s"], "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": {"workload": base.name, "text": base.text, "realizations_per_step": base.R},
            "factors": out, "clocks": clk}
    print(json.dumps(line))


# --------------------------------------------------------------------- graph
def run_graph(args):
    """The workload's per-realization path (sampler with lognormal + Poisson,
    both power spectra with mean and covariance) as replays of one captured
    plan; the embedding is computed once before the timed region (step a2 is
    one-time per spectrum).  Each replay draws new realizations."""
    import torch

    from paper_1406_6072_gb300 import cf
    from paper_1406_6072_gb300 import workloads as W
    from paper_1406_6072_gb300.pipeline import FieldPipeline
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wl = W.CONFIGS[args.workload]
    stream = torch.cuda.Stream(dev)
    pipe = FieldPipeline(wl, dev, stream=stream)
    R = pipe.R
    with torch.cuda.stream(stream):
        pipe.embed()
        lp = cf.make_lp(wl.sigma2, wl.nbar, pipe.counts, wl.seed + 1000) if pipe.with_lp else None
        kw = {}
        if pipe.with_pk:
            kw = dict(bins=pipe.bins, pk=pipe.pk, nmodes=pipe.nmodes, mean=pipe.mean, cov=pipe.cov)
            if pipe.with_lp:
                kw.update(pk_counts=pipe.pkg, mean_counts=pipe.meang, cov_counts=pipe.covg)
        plan = cf.Plan(pipe.emb, wl.seed, 0, R, pipe.fields, lp=lp, stream=stream, **kw)
        for _ in range(args.warmup):
            plan.launch(stream)
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            plan.launch(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    plan.close()
    line = {"metric": METRIC + " (graph replay, embedding cached)", "value": pipe.cells_per_step / (ms * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "text": wl.text, "realizations_per_step": R,
                       "realizations_per_s": R / (ms * 1e-3), "mode": "cf_plan replay"},
            "clocks": clk}
    print(json.dumps(line))


# --------------------------------------------------------------------- small requests
def run_small_requests(args):
    """Launch-bound small requests (the serving mix's 64^2 and 32^3 surveys):
    binary32 sampler + lognormal/Poisson per call, with one launch per pass
    (the default), as one persistent cooperative launch (cf_tune_set), and as
    the replay of a captured plan; per call: device time (back-to-back calls,
    CUDA events) and latency (each call synchronised, host clock)."""
    import numpy as np
    import torch

    from paper_1406_6072_gb300 import cf
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    calls = max(50, args.steps)
    out = {}
    with torch.cuda.stream(stream):
        for n, R in (((64, 64), 1), ((64, 64), 8), ((32, 32, 32), 1), ((32, 32, 32), 8)):
            emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 4.0), cf.CF_EMBED_CLAMP, stream)
            fields = torch.empty((R, 2) + n, dtype=torch.float32, device=dev)
            counts = torch.empty((R, 2) + n, dtype=torch.int32, device=dev)
            lp = cf.make_lp(1.0, 2.0, counts, 9)
            row = {}
            for mode in ("per_pass", "persistent", "graph"):
                cf.cf_tune_set(emb, cf.CF_F32, 0, 0, 0, 1 if mode == "persistent" else 0)
                wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
                ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=dev)
                plan = cf.Plan(emb, 1, 0, R, fields, lp=lp, stream=stream) if mode == "graph" else None

                def call(k):
                    if plan is not None:
                        plan.launch(stream)
                    else:
                        cf.cf_sample_lp(emb, 1, R * k, R, cf.CF_F32, fields, lp, ws, wsb, stream)

                for k in range(args.warmup + 3):
                    call(k)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for k in range(calls):
                    call(k)
                e1.record(stream)
                torch.cuda.synchronize()
                dev_us = 1e3 * e0.elapsed_time(e1) / calls
                lat = []
                for k in range(calls):
                    t0 = time.perf_counter()
                    call(k)
                    stream.synchronize()
                    lat.append(1e6 * (time.perf_counter() - t0))
                row[mode] = {"us_per_call_back_to_back": round(dev_us, 2),
                             "latency_us_p50": round(float(np.percentile(lat, 50)), 2),
                             "latency_us_p99": round(float(np.percentile(lat, 99)), 2)}
                if plan is not None:
                    plan.close()
                del ws
            cf.cf_tune_set(emb, cf.CF_F32)
            emb.close()
            out["%s R=%d" % ("x".join(map(str, n)), R)] = row
    best = min(v["per_pass"]["us_per_call_back_to_back"] / v["persistent"]["us_per_call_back_to_back"]
               for v in out.values())
    line = {"metric": "small-request sampler calls: one launch per pass vs one persistent launch vs graph replay",
            "value": best, "unit": "speed-up of the persistent launch (smallest over the shapes)", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "small_requests", "calls": calls,
                       "text": "2D 64^2 (embedded 128^2) and 3D 32^3 (64^3) Gaussian xi, 1 or 8 realizations, "
                               "lognormal + Poisson nbar = 2"},
            "results": out}
    print(json.dumps(line))


# --------------------------------------------------------------------- serving
def run_serving(args):
    """Mixed request stream through cf_serve_* (continuous batching), against
    the sequential one-request-at-a-time binary64 path (cf_embed + cf_sample
    in binary64, synchronised per request) on a 200-request subsample."""
    import threading as th

    import numpy as np
    import torch

    from paper_1406_6072_gb300 import cf
    from paper_1406_6072_gb300 import workloads as W
    torch.cuda.set_device(0)
    base = W.serving_requests(args.serve_requests, seed=5, rate_hz=1.0)

    def req_of(q):
        return cf.make_request(q["n"], q["xi_kind"], q["amp"], q["scale"], q["beta"], seed=q["seed"], r0=0, R=q["R"],
                               embed_flags=cf.CF_EMBED_CLAMP)

    def serve(reqs, rate):
        sv = cf.cf_serve_create(cf.make_serve_cfg(max_inflight=4, cache_entries=96, max_batch_realizations=256,
                                                  hbm_budget=96 << 30, small_request_cells=1 << 20))
        tickets = []
        lock = th.Lock()
        done_flag = [False]

        parts = []  # (latency, queue, run, cache hit, output cells) per request
        work = {}   # ticket -> output cells (2 R prod n)

        def waiter():
            k = 0
            clamped = 0
            while True:
                with lock:
                    if k >= len(tickets):
                        if done_flag[0]:
                            break
                        t = None
                    else:
                        t = tickets[k]
                if t is None:
                    time.sleep(1e-4)
                    continue
                r = cf.cf_serve_wait(sv, t, -1)
                clamped += r["embed"]["clamped"]
                if r["status"] == cf.CF_OK:
                    parts.append((r["latency_ms"], r["queue_ms"], r["run_ms"], r["cache_hit"], work[t]))
                cf.cf_serve_release(sv, t)
                k += 1
            waiter.clamped = clamped

        w = th.Thread(target=waiter)
        w.start()
        t0 = time.perf_counter()
        for q in reqs:
            if rate:
                delay = t0 + q["t_arrival"] / rate - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            tk = cf.cf_serve_submit(sv, req_of(q))
            with lock:
                work[tk] = 2 * q["R"] * int(np.prod(q["n"]))
                tickets.append(tk)
        with lock:
            done_flag[0] = True
        w.join()
        wall = time.perf_counter() - t0
        st = cf.cf_serve_stats(sv)
        cf.cf_serve_destroy(sv)
        st["wall_s"] = wall
        st["clamped_requests"] = waiter.clamped
        # where the time goes: queueing (waiting for a slot, memory or the
        # spectrum's build) against running, and cache hits against misses
        a = np.asarray(parts, dtype=np.float64).reshape(-1, 5)
        pct = lambda x, q: float(np.percentile(x, q)) if x.size else None
        hit, miss = a[a[:, 3] == 1], a[a[:, 3] == 0]
        # requests span 4 orders of magnitude of work (64^2 x 1 to 128^3 x 32
        # realizations): latency per class of output cells
        classes = {}
        for name, lo, hi in (("small <1M cells", 0, 1 << 20), ("medium 1M-16M", 1 << 20, 1 << 24),
                             ("large >=16M", 1 << 24, 1 << 62)):
            c = a[(a[:, 4] >= lo) & (a[:, 4] < hi)]
            classes[name] = {"requests": int(c.shape[0]), "p50_ms": pct(c[:, 0], 50), "p99_ms": pct(c[:, 0], 99),
                             "p99_queue_ms": pct(c[:, 1], 99)}
        st["attribution"] = {"p50_queue_ms": pct(a[:, 1], 50), "p99_queue_ms": pct(a[:, 1], 99),
                             "p50_run_ms": pct(a[:, 2], 50), "p99_run_ms": pct(a[:, 2], 99),
                             "p99_ms_cache_hit": pct(hit[:, 0], 99), "p99_ms_cache_miss": pct(miss[:, 0], 99),
                             "p50_ms_cache_miss": pct(miss[:, 0], 50),
                             "miss_fraction": float(miss.shape[0] / max(1, a.shape[0])), "by_work": classes}
        return st

    n_cap = min(1000, len(base))
    cap = serve(base[:n_cap], None)   # closed loop: everything at once
    cap_rps = cap["completed"] / cap["wall_s"]
    rates = {}
    per = max(1, (len(base) - n_cap) // 4)
    for i, f in enumerate((0.5, 0.8, 1.0, 1.2)):
        chunk = base[n_cap + i * per: n_cap + (i + 1) * per]
        t_first = chunk[0]["t_arrival"]
        chunk = [dict(q, t_arrival=q["t_arrival"] - t_first) for q in chunk]
        st = serve(chunk, f * cap_rps)
        rates["%.1fx" % f] = {"offered_req_per_s": f * cap_rps, "completed": st["completed"],
                              "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                              "realizations_per_s": st["realizations_per_s"], "batches": st["batches"],
                              "batched_requests": st["batched_requests"], "cache_hits": st["cache_hits"],
                              "cache_misses": st["cache_misses"], "peak_gb": st["bytes_peak"] / 1e9,
                              "clamped_requests": st["clamped_requests"], "attribution": st["attribution"]}
    # sequential binary64 path on a subsample
    rng = np.random.default_rng(7)
    sub = [base[i] for i in rng.choice(len(base), size=min(200, len(base)), replace=False)]
    lat, reals = [], 0
    t_all = time.perf_counter()
    for q in sub:
        t1 = time.perf_counter()
        emb = cf.cf_embed(cf.make_grid(q["n"]), cf.make_xi(q["xi_kind"], q["amp"], q["scale"], q["beta"]),
                          cf.CF_EMBED_CLAMP)
        wsb = cf.cf_sample_workspace_size(emb, q["R"], cf.CF_F64)
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device="cuda:0")
        out = torch.empty((q["R"], 2) + tuple(q["n"]), dtype=torch.float64, device="cuda:0")
        cf.cf_sample(emb, q["seed"], 0, q["R"], cf.CF_F64, out, ws, wsb)
        torch.cuda.synchronize()
        emb.close()
        lat.append(1e3 * (time.perf_counter() - t1))
        reals += q["R"]
        del out, ws
    seq_wall = time.perf_counter() - t_all
    lat = np.sort(np.asarray(lat))
    served = rates["1.0x"]
    # CPU baseline: the oracle, one request at a time, on the same subsample
    # (in order) until 30 s have passed; realizations/s over what it finished
    import oracle
    oracle.build()
    o_reals, o_done, t_o = 0, 0, time.perf_counter()
    for q in sub:
        e = oracle.embed(list(q["n"]), q["xi_kind"], q["amp"], q["scale"], q["beta"], clamp=True)
        oracle.sample(q["n"], e["sqrt_lambda"], q["seed"], 0, q["R"], 0)
        o_reals += q["R"]
        o_done += 1
        if time.perf_counter() - t_o > 30.0:
            break
    o_wall = time.perf_counter() - t_o
    line = {"metric": "served realizations/s, mixed 2D/3D request stream (Poisson arrivals at capacity)",
            "value": served["realizations_per_s"], "unit": "realizations/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving", "requests": len(base), "capacity_req_per_s": cap_rps,
                       "capacity_realizations_per_s": cap["realizations_per_s"],
                       "text": "2D sides 64..1024 and 3D sides 32..128, gaussian / generalised-Cauchy xi, amp "
                               "U(0.2,1.5), scale in {2,..,16}, 1-32 realizations, clamping allowed, seed 5"},
            "p50_ms": served["p50_ms"], "p99_ms": served["p99_ms"], "rates": rates,
            "sequential_f64": {"requests": len(sub), "realizations_per_s": reals / seq_wall,
                               "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                               "note": "one request at a time: cf_embed + binary64 cf_sample, synchronised"},
            "cpu_baseline": {"value": o_reals / o_wall, "unit": "realizations/s", "cores": 1, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": "the first %d requests of the same 200-request subsample (%d realizations), "
                                       "embedding + binary64 fields per request, %.1f s" % (o_done, o_reals, o_wall)}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------- our arm
def e2e_run(pipe, wl, steps, warmup, rank, world=1):
    """Same metric through the public API with host buffers: each step copies
    the xi table from pinned host memory, embeds it, samples, computes the
    spectra and reads the fields, counts and spectra back into pinned host
    memory.  Two pipelines on two streams alternate, so that one step's
    device-to-host copies overlap the next step's compute (the host memory of
    each pipeline is reused every other step, after its copies finished)."""
    import numpy as np
    import torch

    import paper_1406_6072_gb300.cf as cf
    from paper_1406_6072_gb300 import replicas
    from paper_1406_6072_gb300.pipeline import FieldPipeline
    m = wl.m
    # The step's input as a user passes it.  2D: the embedded first row of the
    # workload's two-point function tabulated on the host (a measured
    # correlation function), copied in every step.  3D: the analytic xi, whose
    # three parameters travel by value (a 256^3 table would be 134 MB per step).
    table = None
    if len(m) <= 2:
        ax = [np.arange(v) for v in m]
        lag = [np.where(a < n, a, a - 2 * n).astype(np.float64) * c for a, n, c in zip(ax, wl.n, wl.cell)]
        r2 = np.zeros(tuple(int(v) for v in m))
        for a, l in enumerate(lag):
            r2 = r2 + (l ** 2).reshape([-1 if b == a else 1 for b in range(len(m))])
        if wl.xi_kind == cf.CF_XI_GEN_CAUCHY:
            table = wl.amp / (1.0 + r2 / wl.scale ** 2) ** wl.beta
        elif wl.xi_kind == cf.CF_XI_GAUSSIAN:
            table = wl.amp * np.exp(-r2 / (2.0 * wl.scale ** 2))
        elif wl.xi_kind == cf.CF_XI_EXPONENTIAL:
            table = wl.amp * np.exp(-np.sqrt(r2) / wl.scale)
        else:
            return None
    h_table = torch.from_numpy(np.ascontiguousarray(table)).pin_memory() if table is not None else None
    other = FieldPipeline(wl, pipe.dev, stream=torch.cuda.Stream(pipe.dev), fused=pipe.fused,
                          embed_df=bool(pipe.flags & cf.CF_EMBED_DF))
    lanes = []
    for p in (pipe, other):
        if h_table is not None:
            d_table = torch.empty_like(h_table, device=p.dev)
            xi = cf.make_xi(cf.CF_XI_TABLE, table=d_table, table_on_device=1)
        else:
            d_table = None
            xi = cf.make_xi(wl.xi_kind, wl.amp, wl.scale, wl.beta)
        # every result the step computes: fields, counts, both spectra with
        # their mean and covariance (those of the pipeline's configuration)
        outs = [o for o in (getattr(p, a, None) for a in ("fields", "counts", "pk", "mean", "cov", "pkg",
                                                           "meang", "covg")) if o is not None]
        h_outs = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]
        lanes.append({"p": p, "d_table": d_table, "outs": outs, "h_outs": h_outs, "xi": xi,
                      "copy": torch.cuda.Stream(p.dev), "computed": torch.cuda.Event(),
                      "done": torch.cuda.Event()})

    def one(k):
        # lane k % 2: table in, embed, sample, spectra on its compute stream;
        # results out on its copy stream, so that its next embedding does not
        # queue behind them; its next sampling waits (on the device) until the
        # copies have read the previous results
        ln = lanes[k % 2]
        p = ln["p"]
        if h_table is not None:
            with torch.cuda.stream(p.embed_stream):
                ln["d_table"].copy_(h_table, non_blocking=True)  # read by the embedding, in its stream order
        with torch.cuda.stream(p.stream):
            p.embed(ln["xi"])
            p.stream.wait_event(ln["done"])
            p.sample(r0=replicas.realization_start(rank, world, k, p.R))
            p.spectra()
            ln["computed"].record(p.stream)
        with torch.cuda.stream(ln["copy"]):
            ln["copy"].wait_event(ln["computed"])
            for h, d in zip(ln["h_outs"], ln["outs"]):
                h.copy_(d, non_blocking=True)
            ln["done"].record(ln["copy"])

    for k in range(warmup):
        one(k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        one(1000 + k)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    other.close()
    h2d = h_table.numel() * 8 if h_table is not None else 0
    d2h = sum(h.numel() * h.element_size() for h in lanes[0]["h_outs"])
    return ms, h2d, d2h, ("tabulated xi, %d doubles copied in per step" % h_table.numel()) if h_table is not None \
        else "analytic xi (parameters by value)"


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "small_requests":
        return run_small_requests(args)
    if args.workload.endswith("_sweep"):
        return run_sweep(args)
    if args.workload == "cauchy2d_n512_padding":
        return run_padding(args)
    if args.graph:
        return run_graph(args)
    if args.workload == "mock_n128":
        return run_mock(args)
    import torch

    from paper_1406_6072_gb300 import cf, replicas
    from paper_1406_6072_gb300 import workloads as W
    from paper_1406_6072_gb300.pipeline import FieldPipeline

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = W.CONFIGS[args.workload]
    stream = torch.cuda.Stream(dev)
    # embeddings on their own stream: step k+1's binary64 embedding overlaps
    # step k's sampler and spectra (every step still embeds, samples and
    # computes its spectra; the timed region covers all of it)
    prio = -1 if args.embed_priority == "high" else 0  # lower numbers run first
    pipe = FieldPipeline(wl, dev, stream=stream, embed_stream=torch.cuda.Stream(dev, priority=prio), fused=args.fused,
                         embed_df=args.embed_df)
    R = pipe.R
    # lanes: step k runs on pipeline k % lanes (its own fields, counts,
    # workspaces and streams), so that step k+1's sampler overlaps step k's
    # spectra; every step still embeds, samples and computes both spectra
    lanes = [pipe] + [FieldPipeline(wl, dev, stream=torch.cuda.Stream(dev),
                                    embed_stream=torch.cuda.Stream(dev, priority=prio), fused=args.fused,
                                    embed_df=args.embed_df) for _ in range(max(1, args.lanes) - 1)]

    def run_step(k):
        ln = lanes[k % len(lanes)]
        with torch.cuda.stream(ln.stream):
            ln.step(r0=replicas.realization_start(rank, world, k, R))

    def barrier():
        if dist is not None:
            dist.barrier()

    tuned = None
    if args.tune:
        with torch.cuda.stream(stream):
            pipe.embed()
            chunk, tms = pipe.tune()
            _, rshape, cshape, persist = cf.cf_tune_info(pipe.emb, pipe.dtype)
            tuned = {"chunk": chunk, "rows_shape": rshape, "cols_shape": cshape, "persistent": persist,
                     "ms_per_realization": tms}
    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            run_step(k)
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        cf.cf_kernel_timing(1)
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for ln in lanes[1:]:
            ln.stream.wait_event(e0)
        for k in range(args.steps):
            run_step(args.warmup + k)
        for ln in lanes[1:]:  # the timed region ends when every lane is done
            done = torch.cuda.Event()
            done.record(ln.stream)
            stream.wait_event(done)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        timing = cf.cf_kernel_timing_read()
        cf.cf_kernel_timing(0)
        clk = clocks.stop()
    for ln in lanes[1:]:
        ln.close()
    # the dominant kernel's own duration: inside the timed region its launches
    # share the GPU with the other lane's spectra and the next embedding, so
    # their event times include the time they were held back; timed alone
    # here (the sampler on one stream, nothing else on the device)
    n_alone = 5
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        cf.cf_kernel_timing(1)
        for k in range(n_alone):
            pipe.sample(r0=replicas.realization_start(rank, world, args.warmup + args.steps + k, R))
        torch.cuda.synchronize()
        alone = cf.cf_kernel_timing_read()
        cf.cf_kernel_timing(0)
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = replicas.max_over_ranks(ms, dist, dev)
    cells_all = pipe.cells_per_step * world
    value = cells_all / (ms_max * 1e-3)
    hbm_peak, peak_kind = measured_peaks()
    roof_step, per_kernel = roofline(wl, R, timing, args.steps, hbm_peak, peak_kind, clk.get("sm_mhz"))
    roof, _ = roofline(wl, R, alone, n_alone, hbm_peak, peak_kind, clk.get("sm_mhz"))
    if roof is not None and roof_step is not None:
        roof["timing"] = ("average of %d launches of the kernel timed alone after the timed region (the sampler "
                          "on one stream, nothing else on the device); in_step: its launches inside the timed "
                          "region, overlapped with the other streams' kernels" % n_alone)
        roof["in_step"] = {k: roof_step[k] for k in ("achieved", "frac", "avg_launch_ms", "launches")}
    if roof is not None:
        # the whole step against the scope table's byte counts (the step also
        # embeds and computes both spectra, which these counts leave out)
        floor, plan = step_bytes(wl, R)
        gbs = lambda b: b * R * world / (ms_max * 1e-3) / 1e9
        roof["step"] = {"floor_bytes_per_realization": int(floor), "plan_bytes_per_realization": int(plan),
                        "floor_gbs": round(gbs(floor), 1), "plan_gbs": round(gbs(plan), 1),
                        "floor_frac": round(gbs(floor) / hbm_peak, 4), "plan_frac": round(gbs(plan) / hbm_peak, 4)}
    launches = sum(v[0] for v in per_kernel.values())

    e2e = None
    if not args.no_e2e:
        r = e2e_run(pipe, wl, max(3, args.steps // 2), 2, rank, world)
        if r is not None:
            e_ms, h2d, d2h, e_input = r
            e_max = replicas.max_over_ranks(e_ms, dist, dev)
            e2e = {"value": cells_all / (e_max * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(d2h), "ms_per_step": e_max, "input": e_input}
    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.cpu_sample_realizations)
        cpu_all = cpu_baseline_all_cores(wl, 2)
    cufft = cufft_reference(wl, R, stream) if rank == 0 and not args.no_cufft_reference else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic",
            "config": {"workload": wl.name, "text": wl.text, "realizations_per_step": R * world,
                       "cells_per_step": cells_all, "realizations_per_s": R * world / (ms_max * 1e-3),
                       "l2": "each step writes %d MiB of fields and counts (> 129 MB L2)"
                             % (2 * pipe.cells_per_step * 4 >> 20),
                       "parallelism": "replicas x%d" % world, "tuned_schedule": tuned,
                       "fused_spectra": bool(pipe.fused), "eigenvalue_transforms": "double-float" if args.embed_df
                       else "binary64", "lanes": len(lanes), "embed_priority": args.embed_priority},
            "roofline": roof, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk, "embed_report": pipe.emb.report, "cufft_reference": cufft,
            "kernels": {k: {"launches": v[0], "ms_per_step": v[1] / args.steps} for k, v in sorted(per_kernel.items())},
            "sampler_alone_ms_per_step": {k.split("<")[0]: v[1] / n_alone for k, v in sorted(alone.items())},
        }
        print(json.dumps(line))
    pipe.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
