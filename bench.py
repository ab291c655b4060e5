#!/usr/bin/env python
"""Throughput benchmark of the PDF / alpha_s hot path on GB300.

One step = one pass of the hot path over one batch: x f(x, Q^2) for all 13
flavours (FP64, log-bicubic with continuation outside the grid) plus
alpha_s(Q^2), for 1e7 query points on the three-subgrid synthetic grid.
Metric: evaluations per second (points x flavours, alpha_s counting one per
point).  Inputs (160 MB) and outputs (1.1 GB) exceed the 129 MB L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank evaluates its own batch (weak scaling, no
collective in the data path); the step time is the max over ranks.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import tempfile
import ctypes
import hashlib
import re
import json
import math
import os
import shutil
import subprocess
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "PDF evals/s (points×flavours) FP64 vs FP32 vs surrogate at stated max rel err"
N_POINTS = 10_000_000
MC_EVENTS = 1_000_000
MC_INTEGRATE_EVENTS = 100_000_000
ADJ_POINTS = 1_000_000
SURR_TRAIN, SURR_VAL, SURR_INFER = 20_000_000, 1_000_000, 100_000_000
# PDFFlow Table 2 (Sec. 4.3): all 13 flavours of N_rep members at 2415 x
# points, PDFFlow on a TITAN V or RTX 2080 Ti (system P1), seconds
TABLE2 = {10: 0.07, 50: 0.35, 100: 0.69, 200: 1.46, 300: 1.29, 400: 1.69}
SURR_FLOPS_PER_POINT = 2 * (32 * 128 + 3 * 128 * 128 + 128 * 16)  # padded output layer
SURR_SFU_PER_POINT = 4 * 128  # one hardware tanh per SiLU (features use sincospif on the FMA pipe)
WORKLOAD = ("three Q subgrids (12/15/25 Q knots split at Q = 1.51 and 4.92 GeV, Q in [1, 1e5] GeV), "
            "196 x knots in [1e-9, 1], 13 flavours; 1e7 queries per rank, x log-uniform in [1e-10, 1], "
            "Q log-uniform in [1, 2e5] GeV (15% outside the grid); all flavours + alpha_s per point")

# Ceilings.  FP64/FP32 FMA: GB300 has 152 SMs at up to 2070 MHz; FP64 issues
# 2 DFMA/clk/SM (1.25 TFLOP/s nominal), FP32 128 FFMA/clk/SM.
SMS, SM_MHZ = 152, 2070.0
FP64_PEAK = SMS * 2 * 2 * SM_MHZ * 1e6       # flop/s
FP32_PEAK = SMS * 128 * 2 * SM_MHZ * 1e6

# Algorithmic work per evaluation (flops): the separable 4x4 contraction is
# 16 multiply-adds (32 flops) per site; each point also costs 2 logs and
# ~40 flops of Hermite/tangent weights.  Continuation rules: a log-linear
# pair rule is 5 ops (div, log, mul, exp, mul), the low-Q^2 rule 9.
FLOP_SITE, FLOP_POINT, FLOP_PAIR, FLOP_LOWQ = 32, 42, 5, 9
CLASS_EVAL_FLOPS = {  # class -> flops per (point, flavour) beyond the point part
    "in": 1 * FLOP_SITE,
    "lowx": 2 * FLOP_SITE + FLOP_PAIR,
    "highq": 2 * FLOP_SITE + FLOP_PAIR,
    "lowq": 2 * FLOP_SITE + FLOP_LOWQ,
    "lowx_highq": 4 * FLOP_SITE + 3 * FLOP_PAIR,
    "lowx_lowq": 4 * FLOP_SITE + 2 * FLOP_LOWQ + FLOP_PAIR,
}


def classify(g, x, q2):
    """Class counts of a batch (host-side bookkeeping for the flop count)."""
    lowx = x < g.x_knots[0]
    lowq = q2 < g.q2_knots[0]
    highq = q2 > g.q2_knots[-1]
    return {
        "in": int((~lowx & ~lowq & ~highq).sum()),
        "lowx": int((lowx & ~lowq & ~highq).sum()),
        "highq": int((~lowx & highq).sum()),
        "lowq": int((~lowx & lowq).sum()),
        "lowx_highq": int((lowx & highq).sum()),
        "lowx_lowq": int((lowx & lowq).sum()),
    }


def algorithmic_flops(counts, nflav):
    return sum(c * (FLOP_POINT + nflav * CLASS_EVAL_FLOPS[k]) for k, c in counts.items())


# the translation units each captured kernel is built from, with everything
# they include from the package (a capture counts only while all are unchanged)
KERNEL_SOURCES = {
    "k_xf64<points> near + far": ("xf64.cu", "grid.cu"),
    "k_xf32<points>": ("xfxq2.cu", "grid.cu"),
}
_INCLUDE_RE = re.compile(r'^\s*#\s*include\s+"([^"]+)"', re.M)


def kernel_source_files(kernel):
    dirs = (ROOT / "paper_2009_06635_gb300" / "csrc", ROOT / "include")
    seen, todo = [], list(KERNEL_SOURCES[kernel])
    while todo:
        name = todo.pop(0)
        path = next((d / name for d in dirs if (d / name).exists()), None)
        if path is None or path in seen:
            continue
        seen.append(path)
        todo.extend(_INCLUDE_RE.findall(path.read_text()))
    return seen


def kernel_source_hash(kernel="k_xf64<points> near + far"):
    h = hashlib.sha256()
    for path in kernel_source_files(kernel):
        h.update(path.read_bytes())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, n_points):
    """DRAM bytes per launch from the committed ncu summary, or None if the
    kernel source changed since the counters were taken."""
    f = ROOT / "profiles" / "traffic.json"
    if not f.exists():
        return None
    try:
        rec = json.loads(f.read_text()).get(kernel)
    except Exception:
        return None
    if not rec or rec.get("source_hash") != kernel_source_hash(kernel):
        return None
    return rec["dram_bytes_per_point"] * n_points


def profiled_pipes(kernel):
    """Per-point busy time of each SM unit for `kernel` (all its launches of
    one call), from the committed ncu capture (profiles/pipes.json), or None
    if the source changed since."""
    f = ROOT / "profiles" / "pipes.json"
    if not f.exists():
        return None
    try:
        rec = json.loads(f.read_text()).get(kernel)
    except Exception:
        return None
    if not rec or rec.get("source_hash") != kernel_source_hash(kernel):
        return None
    return rec


def unit_bound(pipes, n, sm_mhz, alg_bytes, hbm_gbs):
    """Seconds each unit needs for n points at its full rate: the capture's
    busy time per point of every SM unit (its utilisation times the launch
    duration, summed over the call's launches), scaled from the capture's SM
    clock to this run's; HBM from the algorithmic bytes over the measured copy
    bandwidth.  Returns {unit: seconds}."""
    scale = pipes["sm_mhz"] / sm_mhz
    t = {u: s * n * scale for u, s in pipes["per_point_busy_s"].items()}
    t["hbm"] = alg_bytes / (hbm_gbs * 1e9)
    return t


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = Path(tempfile.gettempdir()) / f"pdf_gb300_clocks_{os.getpid()}.csv"

    def start(self):
        if not shutil.which("nvidia-smi"):
            return
        self.path.parent.mkdir(exist_ok=True)
        self.fh = open(self.path, "w")
        self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits", "-lms", "50"],
                                     stdout=self.fh, stderr=subprocess.DEVNULL)
        time.sleep(0.5)  # let the sampler start before the measured work

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = [r.split(", ") for r in self.path.read_text().strip().splitlines() if r.strip()]
        rows = [r for r in rows if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


def _cpulist(text):
    cpus = set()
    for part in text.strip().split(","):
        if part:
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
    return cpus


class near_gpu:
    """Within the block the process runs on the CPUs of the GPU's NUMA node
    (read from sysfs), so pages first touched there are that node's memory;
    the previous affinity comes back on exit.  Records what it found."""

    def __init__(self, local):
        self.local = local
        self.info = {"gpu_pci": None, "gpu_numa_node": None, "cpus_used": None}
        self.saved = None

    def __enter__(self):
        import torch

        try:
            pr = torch.cuda.get_device_properties(self.local)
            bdf = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
            self.info["gpu_pci"] = bdf
            node = int(Path(f"/sys/bus/pci/devices/{bdf}/numa_node").read_text())
            self.info["gpu_numa_node"] = node
            if node >= 0 and hasattr(os, "sched_setaffinity"):
                cpus = _cpulist(Path(f"/sys/devices/system/node/node{node}/cpulist").read_text())
                self.saved = os.sched_getaffinity(0)
                use = self.saved & cpus
                if use:
                    os.sched_setaffinity(0, use)
                    self.info["cpus_used"] = len(use)
                else:
                    self.saved = None
        except Exception as e:  # no sysfs entry, no permission: run where we are
            self.info["note"] = f"placement not applied: {type(e).__name__}"
        return self.info

    def __exit__(self, *exc):
        if self.saved is not None:
            os.sched_setaffinity(0, self.saved)
        return False


def buffer_nodes(tensor):
    """NUMA nodes holding a host tensor's pages ({node: pages}), from /proc/self/numa_maps."""
    addr = tensor.data_ptr()
    try:
        best = None
        for line in Path("/proc/self/numa_maps").read_text().splitlines():
            f = line.split()
            start = int(f[0], 16)
            if start <= addr and (best is None or start > best[0]):
                best = (start, f)
        if best is None:
            return None
        return {k[1:].split("=")[0]: int(k.split("=")[1]) for k in best[1] if k.startswith("N") and "=" in k}
    except Exception:
        return None


def link_rates(dev, hbuf_out, hbuf_in, sync, reps=5):
    """Host-link rates (GB/s) on the given pinned buffers: device to host into
    hbuf_out, host to device from hbuf_in; best of `reps` timed copies each
    after a warm copy, CUDA events on the current stream."""
    import torch

    res = {}
    for name, dst, src in (("d2h_gbs", hbuf_out, torch.empty_like(hbuf_out, device=dev)),
                           ("h2d_gbs", torch.empty_like(hbuf_in, device=dev), hbuf_in)):
        dst.copy_(src, non_blocking=True)
        sync()
        best = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dst.copy_(src, non_blocking=True)
            b.record()
            sync()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        res[name] = src.numel() * src.element_size() / (best * 1e-3) / 1e9
        del dst, src
    return res


def dist_setup():
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_timed(fn, steps, warmup, world, sync):
    """W untimed steps, then K steps bracketed by barrier + synchronize."""
    import torch

    for _ in range(warmup):
        fn()
    sync()
    barrier(world)
    sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    sync()
    barrier(world)
    sync()
    return e0.elapsed_time(e1) / steps  # ms per step


# --------------------------------------------------------------------------
# reference arm: the CPU oracle on the host cores
# --------------------------------------------------------------------------

def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2009_06635_gb300 import synthetic as S

    g = S.grid_full()
    og = oracle.OracleGrid(g)
    sample = 200_000
    x, q2 = S.queries_full(sample, 3)
    for _ in range(max(1, args.warmup)):
        og.xfxq2(x[:20_000], q2[:20_000])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        og.xfxq2(x, q2)
        og.alphas(q2)
    dt = (time.perf_counter() - t0) / args.steps
    evals = sample * (g.nflav + 1)
    value = evals / dt
    cores = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference_sample_points_per_step": sample},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} points of the same query law per step, all flavours + alpha_s"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def cpu_baseline_leg(g, x, q2, out_gpu, a_gpu, x32, q32, out32, target_s=10.0):
    """Time the oracle as it stands on the host cores on a bounded sample of
    the workload; with the same oracle outputs, state the GPU paths' errors
    on that sample."""
    import oracle

    og = oracle.OracleGrid(g)
    cores = oracle.max_threads()
    probe = 20_000
    t0 = time.perf_counter()
    og.xfxq2(x[:probe], q2[:probe])
    og.alphas(q2[:probe])
    per_pt = (time.perf_counter() - t0) / probe
    m = int(min(len(x), max(probe, target_s / per_pt)))
    idx = np.random.default_rng(11).choice(len(x), m, replace=False)
    idx.sort()
    t0 = time.perf_counter()
    v, s, fl = og.xfxq2(x[idx], q2[idx])
    av, asv = og.alphas(q2[idx])
    dt = time.perf_counter() - t0
    rate = m * (g.nflav + 1) / dt
    # the same oracle on one host core, on the first tenth of the sample
    m1 = max(probe, m // 10)
    t0 = time.perf_counter()
    og.xfxq2(x[idx[:m1]], q2[idx[:m1]], nthreads=1)
    og.alphas(q2[idx[:m1]], nthreads=1)
    rate1 = m1 * (g.nflav + 1) / (time.perf_counter() - t0)
    err64 = np.abs(out_gpu[idx] - v) / np.maximum(np.abs(v), s)
    err64 = np.where(fl, 0.0, err64)
    # the paper's eq. (1) on the same outputs, leaving out those at a zero
    # crossing of xf (|oracle| below 1e-3 of the data mass)
    far = ~fl & (np.abs(v) >= 1e-3 * s)
    eq1 = np.where(far, np.abs(out_gpu[idx] - v) / (np.abs(v) + 1e-16), 0.0)
    xs, qs = x[idx], q2[idx]
    ingrid = (xs >= g.x_knots[0]) & (q2[idx] >= g.q2_knots[0]) & (qs <= g.q2_knots[-1])
    above = eq1 > 1e-12
    aerr = float((np.abs(a_gpu[idx] - av) / np.maximum(np.abs(av), asv)).max())
    # FP32 path against the oracle at the float inputs (a sub-sample)
    k = min(m, 200_000)
    v3, s3, f3 = og.xfxq2(x32[idx[:k]].astype(np.float64), q32[idx[:k]].astype(np.float64))
    err32 = np.where(f3, 0.0, np.abs(out32[idx[:k]] - v3) / np.maximum(np.abs(v3), s3))
    return ({"value": rate, "unit": "evals/s", "cores": cores, "kind": "oracle",
             "sample": f"{m} of the {len(x)} points (all flavours + alpha_s), {dt:.1f} s on {cores} threads",
             "one_core": {"value": rate1, "unit": "evals/s", "sample": f"{m1} of those points on 1 thread"}},
            {"fp64_max_scaled_err": float(np.nanmax(err64)), "alphas_max_scaled_err": aerr,
             "fp64_eq1_max_per_flavour": [float(e) for e in eq1.max(axis=0)],
             "eq1": "|gpu - oracle| / (|oracle| + 1e-16), paper eq. (1), per flavour",
             "eq1_near_zero_excluded": int((~fl & ~far).sum()),
             "eq1_max_in_grid": float(eq1[ingrid].max()) if ingrid.any() else 0.0,
             "eq1_max_continued": float(eq1[~ingrid].max()) if (~ingrid).any() else 0.0,
             "eq1_outputs_above_1e-12": int(above.sum()),
             "eq1_above_1e-12_median_mass_over_value": float(np.median((s / np.maximum(np.abs(v), 1e-300))[above]))
             if above.any() else None,
             "fp32_max_scaled_err_per_flavour": [float(e) for e in np.nanmax(err32, axis=0)],
             "scaled_err": "|gpu - oracle| / max(|oracle|, sum|w f|), on the sampled points",
             "marginal_excluded": int(fl.sum()), "sample_points": m})


def small_grid_leg(dev, sync, reps=200):
    """The single-subgrid workload (50 x 40 knots, 11 flavours, 1e4 in-grid
    queries): latency-dominated, so the time of one call matters; FP64 and
    FP32 all flavours + alpha_s, device buffers, CUDA events around `reps`
    back-to-back calls after a warm-up."""
    import torch

    import paper_2009_06635_gb300 as P
    from paper_2009_06635_gb300 import synthetic as S

    g = S.grid_single_subgrid()
    G = P.pdf_load_grid(g)
    x, q2 = S.queries_single_subgrid(10_000, 2)
    n, nf = len(x), g.nflav
    res = {"workload": "single subgrid: 50 x knots in [1e-7, 1], 40 Q^2 knots in [2.7, 1e8], 11 flavours; "
                       "1e4 in-grid queries (seed 2)", "points": n}
    for tag, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        xd, qd = torch.from_numpy(x).to(dev, dt), torch.from_numpy(q2).to(dev, dt)
        out = torch.empty((n, nf), dtype=dt, device=dev)
        aout = torch.empty((n,), dtype=dt, device=dev)
        for _ in range(10):
            P.xfxq2_all_flavours_alphas(G, xd, qd, out=out, alphas_out=aout)
        sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            P.xfxq2_all_flavours_alphas(G, xd, qd, out=out, alphas_out=aout)
        b.record()
        sync()
        us = a.elapsed_time(b) / reps * 1e3
        res[tag] = {"us_per_call": us, "value": n * (nf + 1) / (us * 1e-6), "unit": "evals/s"}
    return res


def surrogate_leg(args, G, g, dev, world, sync, rank, nf, ms_per_eval64, target="envelope"):
    """Learned surrogate: train on 2e7 in-grid samples, map its error against
    the FP64 interpolator on 1e6 validation points, infer on 1e8 points.
    target: "residual" (xf = B + 2^-10 E(x) y, B a bilinear base table),
    "envelope" (xf = E(x) y) or "asinh" (xf = c sinh y)."""
    import torch

    from paper_2009_06635_gb300 import synthetic as S
    from paper_2009_06635_gb300.surrogate import Surrogate

    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    s = Surrogate(G, max_batch=8192, target=target)
    xt, qt = S.ingrid_samples(g, SURR_TRAIN, 7 + 1000 * rank)
    xtd, qtd = torch.from_numpy(xt).to(dev), torch.from_numpy(qt).to(dev)
    del xt, qt
    steps = 2 * SURR_TRAIN // 8192
    sync()
    t0 = time.perf_counter()
    final_loss = s.train(G, xtd, qtd, batch=8192, steps=steps, lr=2e-3, lr_min=1e-5, warmup=200)
    sync()
    train_s = time.perf_counter() - t0
    del xtd, qtd
    xv, qv = S.ingrid_samples(g, SURR_VAL, 11 + 1000 * rank)
    stats = s.build_error_map(G, torch.from_numpy(xv).to(dev), torch.from_numpy(qv).to(dev), threshold=1e-3)
    xi, qi = S.ingrid_samples(g, SURR_INFER, 8 + 1000 * rank)
    xid, qid = torch.from_numpy(xi).to(dev), torch.from_numpy(qi).to(dev)
    del xi, qi
    out = torch.empty((SURR_INFER, nf), dtype=torch.float32, device=dev)
    ev = []

    def step():
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        s.eval(xid, qid, out=out)
        b.record()
        ev.append((a, b))

    ms = run_timed(step, max(3, args.steps // 10), 2, world, sync)
    kms = float(np.mean([a.elapsed_time(b) for a, b in ev[2:]]))
    # accuracy of the network alone on 1e6 of the inference points, against the interpolator
    k = 1_000_000
    ref = P_xf(G, xid[:k], qid[:k])
    net = out[:k].double()
    scale = torch.from_numpy(1e-5 * np.abs(g.values).reshape(-1, nf).max(axis=0)).to(dev)
    err = ((net - ref).abs() / torch.maximum(ref.abs(), scale)).max(dim=0).values.cpu().numpy()
    perr = ((net - ref).abs() / torch.maximum(ref.abs(), scale)).max(dim=1).values
    within = float((perr <= 1e-3).float().mean())
    within2 = float((perr <= 1e-2).float().mean())
    q = [float(v) for v in torch.quantile(perr[:100_000].float(), torch.tensor([0.5, 0.9, 0.99], device=dev))]
    fb_out, nfb = s.eval_fallback(G, xid[:k], qid[:k])
    served = (fb_out != ref).any(dim=1)
    ferr = ((fb_out - ref).abs() / torch.maximum(ref.abs(), scale))[served]
    served_err = ferr.max(dim=0).values.cpu().numpy() if ferr.shape[0] else np.zeros(nf)
    sync()
    t0 = time.perf_counter()
    for _ in range(3):
        s.eval_fallback(G, xid, qid)
    sync()
    fb_s = (time.perf_counter() - t0) / 3
    flops = SURR_FLOPS_PER_POINT * SURR_INFER
    sfu_peak = SMS * 16 * SM_MHZ * 1e6
    return {
        "value": world * SURR_INFER * nf / (ms * 1e-3), "unit": "evals/s (network only)", "ms_per_step": ms,
        "points": SURR_INFER, "train": {"samples": SURR_TRAIN, "steps": steps, "batch": 8192, "seconds": train_s,
                                        "final_loss": final_loss},
        "error_map": stats,
        "max_rel_err_per_flavour": [float(e) for e in err],
        "rel_err": "|net - interp| / max(|interp|, 1e-5 max|xf_f|), network alone, 1e6 inference points",
        "fraction_within_1e-3": within,
        "fraction_within_1e-2": within2,
        "point_max_err_quantiles_50_90_99": q,
        "target": target,
        "fallback": {"threshold": 1e-3, "fallback_fraction": nfb / k, "served_fraction": 1.0 - nfb / k,
                     "value": world * SURR_INFER * nf / fb_s, "unit": "evals/s with fallback (FP64 out)",
                     "gain_vs_fp64_interpolator": (SURR_INFER * nf / fb_s) * ms_per_eval64 * 1e-3,
                     "served_max_rel_err_per_flavour": [float(e) for e in served_err],
                     "note": "each error-map tile is served by the network (residual: plus its base), by the "
                             "residual target's base alone, or by the FP64 interpolator, whichever is within the "
                             "1e-3 threshold on the validation points (the more accurate of the first two); "
                             "errors against the FP64 interpolator on the 1e6 inference points"},
        "gain_vs_fp64_interpolator": (SURR_INFER * nf / (kms * 1e-3)) * ms_per_eval64 * 1e-3,
        "roofline": {"bound": "tensor", "achieved": flops / (kms * 1e-3) / 1e12, "peak": bf16_peak, "unit": "TFLOP/s",
                     "frac": flops / (kms * 1e-3) / 1e12 / bf16_peak,
                     "peak_source": "measured bf16 burst (MEASURED_PEAKS.json)",
                     "sfu_bound_ms": SURR_SFU_PER_POINT * SURR_INFER / sfu_peak * 1e3, "kernel_ms": kms},
    }


def members_leg(args, dev, world, sync, rank):
    """PDFFlow Table 2 workload: 13 flavours x N_rep members x 2415 x points
    (x log-spaced in [1e-9, 1), Q = 1.65 GeV), one launch per N_rep."""
    import torch

    import paper_2009_06635_gb300 as P
    from paper_2009_06635_gb300 import synthetic as S

    g0, vals = S.grid_members(max(TABLE2), seed=12 + 1000 * rank)
    x, q2 = S.fit_points()
    xd, qd = torch.from_numpy(x).to(dev), torch.from_numpy(q2).to(dev)
    rows = []
    for nrep in sorted(TABLE2):
        sync()
        t0 = time.perf_counter()
        G = P.pdf_load_grid(g0, member_values=vals[:nrep])  # host checks, copy, staging kernels (synchronous)
        load_ms = (time.perf_counter() - t0) * 1e3
        out = torch.empty((nrep, len(x), g0.nflav), dtype=torch.float64, device=dev)
        ms = run_timed(lambda: P.xfxq2_all_members(G, xd, qd, out=out), max(5, args.steps // 5), 3, world, sync)
        evals = nrep * len(x) * g0.nflav
        rows.append({"n_rep": nrep, "evals": evals, "ms": ms, "evals_per_s": world * evals / (ms * 1e-3),
                     "load_ms": load_ms,
                     "paper_gpu_s": TABLE2[nrep], "paper_gpu_evals_per_s": evals / TABLE2[nrep]})
        del G, out
    return {"rows": rows, "workload": "13 flavours x N_rep members x 2415 x points (log-spaced in [1e-9, 1)), "
            "Q = 1.65 GeV; members perturb the synthetic set's flavour parameters",
            "paper_hardware": "PDFFlow v1.0 on TITAN V or RTX 2080 Ti (system P1); context, not the target",
            "load_ms": "pdf_load_grid of the N_rep-member set (host validation, host-to-device copy, staging "
                       "kernels), wall clock, once per set; ms is one evaluation call on the loaded set"}


def mc_cut_pass_fraction(x_min, x_max, s, shat_min):
    """Share of events with x1 x2 s >= shat_min for x1, x2 log-uniform in
    [x_min, x_max]: ln x1 + ln x2 has the triangular density of two uniform
    variables on [lo, hi]."""
    lo, hi = math.log(x_min), math.log(x_max)
    span = hi - lo
    a = math.log(shat_min / s) if shat_min > 0 else -math.inf
    if a <= 2 * lo:
        return 1.0
    if a >= 2 * hi:
        return 0.0
    if a <= lo + hi:
        return 1.0 - (a - 2 * lo) ** 2 / (2 * span * span)
    return (2 * hi - a) ** 2 / (2 * span * span)


def mc_leg(G, world, sync, rank, x_max=1.0):
    """Monte Carlo integration (the event workload at full size): 1e8 events per rank in 100
    chunks of 1e6, device RNG, fused PDF + alpha_s load, weights summed on the
    device; the three sums are added over ranks (the integration's one
    exchange step).  Events below the s-hat cut are integrated with weight
    zero and not evaluated; evals_per_s counts the evaluations made."""
    import paper_2009_06635_gb300 as P

    n, chunk = MC_INTEGRATE_EVENTS, MC_EVENTS
    cfg = dict(sqrt_s=13000.0, x_min=1e-6, shat_min=100.0, seed=4)
    P.pdf_mc_integrate(G, cfg["sqrt_s"], cfg["x_min"], cfg["shat_min"], cfg["seed"], 3 * chunk, chunk=chunk)  # warm-up
    sync()
    barrier(world)
    from paper_2009_06635_gb300.sharding import allreduce_mc_sums, mc_event_range

    first, count = mc_event_range(rank, n)
    t0 = time.perf_counter()
    r = P.pdf_mc_integrate(G, cfg["sqrt_s"], cfg["x_min"], cfg["shat_min"], cfg["seed"], count, first_event=first,
                           chunk=chunk)
    sync()
    s = max_over_ranks(world, time.perf_counter() - t0)
    tot = P.McResult(allreduce_mc_sums([r.sum_w, r.sum_w2, r.sum_abs]), world * n)
    passed = mc_cut_pass_fraction(cfg["x_min"], x_max, cfg["sqrt_s"] ** 2, cfg["shat_min"])
    return {"events": world * n, "chunk": chunk, "s": s, "events_per_s": world * n / s,
            "evaluated_fraction": passed, "evals_per_s": world * n * passed * (2 * 13 + 1) / s,
            "estimate": tot.estimate, "std_error": tot.std_error,
            "config": dict(cfg, observable="toy LO: L^2/s-hat [sum_q e_q^2 (q qbar + qbar q) + alpha_s^2 g g]")}


def P_xf(G, x, q2):
    import paper_2009_06635_gb300 as P

    return P.xfxq2_all_flavours(G, x, q2)


def our_arm(args):
    import torch

    import paper_2009_06635_gb300 as P
    from paper_2009_06635_gb300 import _native
    from paper_2009_06635_gb300 import synthetic as S

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sync = torch.cuda.synchronize
    lib = _native.load(build_if_missing=False)

    g = S.grid_full()
    G = P.pdf_load_grid(g)
    n = args.points
    if args.law == "bench":
        x, q2 = S.queries_full(n, 3 + 1000 * rank)
    else:  # one class of point (profiling runs of --only)
        x, q2 = S.queries_class(g, args.law, n, 3 + 1000 * rank)
    counts = classify(g, x, q2)
    nf = g.nflav
    xd = torch.from_numpy(x).to(dev)
    qd = torch.from_numpy(q2).to(dev)
    out = torch.empty((n, nf), dtype=torch.float64, device=dev)
    aout = torch.empty((n,), dtype=torch.float64, device=dev)
    evals_step = n * (nf + 1)

    # per-launch duration of the dominant kernel, on the launching stream
    ev = []

    def step64(record=False):  # one launch: all flavours and alpha_s
        if record:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            P.xfxq2_all_flavours_alphas(G, xd, qd, out=out, alphas_out=aout)
            b.record()
            ev.append((a, b))
        else:
            P.xfxq2_all_flavours_alphas(G, xd, qd, out=out, alphas_out=aout)

    if args.only == "adjoint":  # the adjoint alone on --points points of the same law
        ax, aq, acot = S.adjoint_inputs(n, nf, 5 + 1000 * rank, 6 + 1000 * rank)
        if args.law != "bench":  # points of one class, same cotangents
            ax, aq = S.queries_class(g, args.law, n, 5 + 1000 * rank)
        axd, aqd, acd = torch.from_numpy(ax).to(dev), torch.from_numpy(aq).to(dev), torch.from_numpy(acot).to(dev)
        agx, agq = torch.empty_like(axd), torch.empty_like(aqd)
        agv = torch.zeros((G.nrows, G.nx, nf), dtype=torch.float64, device=dev)
        ms = run_timed(lambda: P.xfxq2_all_flavours_vjp(G, axd, aqd, acd, agx, agq, agv), args.steps, args.warmup,
                       world, sync)
        if rank == 0:
            print(json.dumps({"only": args.only, "points": n, "ms_per_step": ms,
                              "gradients_per_s": n * nf / (ms * 1e-3)}))
        return 0
    if args.only == "surrogate":  # inference alone on in-grid points (its cost does not depend on training)
        from paper_2009_06635_gb300 import synthetic as S
        from paper_2009_06635_gb300.surrogate import Surrogate

        s = Surrogate(G, max_batch=1024, target=args.target)
        xi, qi = S.ingrid_samples(g, n, 8 + 1000 * rank)
        xid, qid = torch.from_numpy(xi).to(dev), torch.from_numpy(qi).to(dev)
        so = torch.empty((n, nf), dtype=torch.float32, device=dev)
        ms = run_timed(lambda: s.eval(xid, qid, out=so), args.steps, args.warmup, world, sync)
        if rank == 0:
            print(json.dumps({"only": args.only, "points": n, "ms_per_step": ms, "evals_per_s": n * nf / (ms * 1e-3),
                              "tflops": SURR_FLOPS_PER_POINT * n / (ms * 1e-3) / 1e12}))
        return 0
    if args.only:
        if args.only == "fp64":
            fn = lambda: P.xfxq2_all_flavours_alphas(G, xd, qd, out=out, alphas_out=aout)  # noqa: E731
        else:
            xs = (xd.float(), qd.float(), out.float(), aout.float())
            fn = lambda: P.xfxq2_all_flavours_alphas(G, xs[0], xs[1], out=xs[2], alphas_out=xs[3])  # noqa: E731
        ms = run_timed(fn, args.steps, args.warmup, world, sync)
        if rank == 0:
            print(json.dumps({"only": args.only, "points": n, "ms_per_step": ms, "evals_per_s": evals_step / (ms * 1e-3)}))
        return 0

    clocks = Clocks(local)
    clocks.start()
    ms64 = run_timed(lambda: step64(True), args.steps, args.warmup, world, sync)
    clk = clocks.stop()
    kern_ms = [a.elapsed_time(b) for a, b in ev[args.warmup:]]
    kern_ms = float(np.mean(kern_ms))
    ms64 = max_over_ranks(world, ms64)
    value = world * evals_step / (ms64 * 1e-3)

    # FP32 path on the same workload
    x32, q32 = x.astype(np.float32), q2.astype(np.float32)
    xd32, qd32 = torch.from_numpy(x32).to(dev), torch.from_numpy(q32).to(dev)
    out32 = torch.empty((n, nf), dtype=torch.float32, device=dev)
    aout32 = torch.empty((n,), dtype=torch.float32, device=dev)
    ev32 = []

    def step32():  # one launch: all flavours and alpha_s
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        P.xfxq2_all_flavours_alphas(G, xd32, qd32, out=out32, alphas_out=aout32)
        b.record()
        ev32.append((a, b))

    ms32 = max_over_ranks(world, run_timed(step32, args.steps, args.warmup, world, sync))
    k32 = float(np.mean([a.elapsed_time(b) for a, b in ev32[args.warmup:]]))

    # single flavour, alpha_s alone, fused MC event batch
    one = torch.empty((n,), dtype=torch.float64, device=dev)
    ms_pid = run_timed(lambda: P.xfxq2(G, 21, xd, qd, out=one), args.steps, 2, world, sync)
    ms_as = run_timed(lambda: P.alphas_q2(G, qd, out=aout), args.steps, 2, world, sync)
    x1, x2, s2 = S.events_mc(MC_EVENTS, 4 + 1000 * rank)
    x1d, x2d = torch.from_numpy(x1).to(dev), torch.from_numpy(x2).to(dev)
    mco = torch.empty((MC_EVENTS, 2 * nf + 1), dtype=torch.float64, device=dev)
    ms_mc = run_timed(lambda: P.pdf_mc_event(G, x1d, x2d, s2, out=mco), args.steps, 2, world, sync)
    x1f, x2f = x1d.float(), x2d.float()
    mco32 = torch.empty((MC_EVENTS, 2 * nf + 1), dtype=torch.float32, device=dev)
    ms_mc32 = run_timed(lambda: P.pdf_mc_event(G, x1f, x2f, float(np.float32(s2)), out=mco32),
                        args.steps, 2, world, sync)

    # adjoint: 1e6 points of the same law, standard-normal cotangents on all
    # flavours; gradients in x, Q^2 and every knot value (zeroed each step)
    ax, aq, acot = S.adjoint_inputs(ADJ_POINTS, nf, 5 + 1000 * rank, 6 + 1000 * rank)
    axd, aqd, acd = torch.from_numpy(ax).to(dev), torch.from_numpy(aq).to(dev), torch.from_numpy(acot).to(dev)
    agx, agq = torch.empty_like(axd), torch.empty_like(aqd)
    agv = torch.zeros((G.nrows, G.nx, nf), dtype=torch.float64, device=dev)

    from paper_2009_06635_gb300.sharding import allreduce_knot_gradient

    def step_adj():  # each rank its own block; the knot gradient is summed over ranks
        agv.zero_()
        P.xfxq2_all_flavours_vjp(G, axd, aqd, acd, agx, agq, agv)
        allreduce_knot_gradient(agv)

    ms_adj = run_timed(step_adj, args.steps, 2, world, sync)

    mc_int = mc_leg(G, world, sync, rank, x_max=float(g.x_knots[-1]))
    small = small_grid_leg(dev, sync)
    members = None if args.no_members else members_leg(args, dev, world, sync, rank)
    surrogate = None if args.no_surrogate else surrogate_leg(args, G, g, dev, world, sync, rank, nf,
                                                             ms64 / (n * (nf + 1)), target="residual")
    surrogate_env = None if args.no_surrogate else surrogate_leg(args, G, g, dev, world, sync, rank, nf,
                                                                 ms64 / (n * (nf + 1)), target="envelope")

    # end to end through the C ABI with host buffers (pinned), copies timed;
    # the buffers are first touched on the GPU's own NUMA node
    with near_gpu(local) as numa:
        hx = torch.from_numpy(x).pin_memory()
        hq = torch.from_numpy(q2).pin_memory()
        hout = torch.empty((n, nf), dtype=torch.float64).pin_memory()
        hal = torch.empty((n,), dtype=torch.float64).pin_memory()
        hout.fill_(0.0)
        hal.fill_(0.0)
    numa["buffer_nodes"] = {k: buffer_nodes(v) for k, v in (("x", hx), ("q2", hq), ("out", hout), ("alphas", hal))}
    e2e_steps = max(3, min(args.steps, 10))
    for _ in range(2):
        P.xfxq2_all_flavours_host(G, hx, hq, out=hout, alphas_out=hal)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        P.xfxq2_all_flavours_host(G, hx, hq, out=hout, alphas_out=hal)
    e2e_s = max_over_ranks(world, (time.perf_counter() - t0) / e2e_steps)
    # the host link on the step's own buffers: best of 5 timed copies each way
    # (after a warm copy), device to host into the output buffer, host to device
    # from the input buffer
    link = link_rates(dev, hout, hx, sync)
    e2e_bound_s = max(8 * n * (nf + 1) / (link["d2h_gbs"] * 1e9), 16 * n / (link["h2d_gbs"] * 1e9))

    # ceilings measured on this GPU
    fp64_meas = ctypes.c_double(0.0)
    fp32_meas = ctypes.c_double(0.0)
    probe = _native.load_probe()
    _native.check_probe(probe.pdf_probe_fma_rate(64, 4096, ctypes.byref(fp64_meas)), "probe fp64")
    _native.check_probe(probe.pdf_probe_fma_rate(32, 65536, ctypes.byref(fp32_meas)), "probe fp32")
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    hbm = peaks.get("hbm_gbs", 6800.0)

    flops = algorithmic_flops(counts, nf)
    achieved = flops / (kern_ms * 1e-3)
    traffic = profiled_traffic("k_xf64<points> near + far", n)
    bytes32 = n * (8 + 4 * nf + 4)  # x, Q^2 in; the flavours and alpha_s out
    alg_bytes = n * (16 + 8 * nf + 8)
    sm_mhz = (clk or {}).get("sm_mhz") or SM_MHZ
    pipes = profiled_pipes("k_xf64<points> near + far")
    if pipes:
        # the kernel's own ceiling: the unit it keeps busiest, at its full rate
        ut = unit_bound(pipes, n, sm_mhz, alg_bytes, hbm)
        binding = max(ut, key=ut.get)
        t_bound = ut[binding]
        roofline = {
            "bound": "hbm" if binding == "hbm" else "alu", "binding_unit": binding,
            "kernel": "xfxq2_all_flavours_alphas FP64 (k_xf64<points> near + far launches, all flavours + alpha_s)",
            "achieved": achieved / 1e12, "peak": flops / t_bound / 1e12, "unit": "TFLOP/s",
            "frac": t_bound / (kern_ms * 1e-3), "traffic": traffic,
            "peak_source": ("per-unit model: each SM unit's busy time per point (ncu utilisation x launch "
                            "duration, both launches of a call, profiles/pipes.json) x points, at the sampled SM "
                            "clock; the peak is the algorithmic flop rate at which the busiest unit is saturated"),
            "unit_ms": {k: v * 1e3 for k, v in ut.items()}, "sm_mhz_used": sm_mhz,
            "kernel_ms": kern_ms, "algorithmic_flops_per_launch": flops,
            "fp64_dfma_peak_tflops": FP64_PEAK / 1e12,
            "fp64_dfma_frac_of_algorithmic_flops": achieved / FP64_PEAK,
            "hbm_frac": alg_bytes / (kern_ms * 1e-3) / (hbm * 1e9)}
    else:  # no capture of this source: the algorithmic bytes against HBM
        roofline = {
            "bound": "hbm", "kernel": "xfxq2_all_flavours_alphas FP64 (k_xf64<points>, all flavours + alpha_s)",
            "achieved": alg_bytes / (kern_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": alg_bytes / (kern_ms * 1e-3) / (hbm * 1e9), "traffic": traffic,
            "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json); no per-unit capture of this source",
            "kernel_ms": kern_ms, "algorithmic_flops_per_launch": flops}
    # FP32: its algorithmic bytes against HBM, and (with a capture of this
    # source) the same per-unit model as the FP64 call
    roofline32 = {"bound": "hbm", "achieved": bytes32 / (k32 * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                  "frac": bytes32 / (k32 * 1e-3) / 1e9 / hbm,
                  "traffic": profiled_traffic("k_xf32<points>", n),
                  "fp32_fma_peak_derived_tflops": FP32_PEAK / 1e12,
                  "fp32_fma_peak_measured_tflops": fp32_meas.value / 1e12}
    pipes32 = profiled_pipes("k_xf32<points>")
    if pipes32:
        ut32 = unit_bound(pipes32, n, sm_mhz, bytes32, hbm)
        b32 = max(ut32, key=ut32.get)
        roofline32["per_unit"] = {
            "binding_unit": b32, "frac": ut32[b32] / (k32 * 1e-3),
            "unit_ms": {k: v * 1e3 for k, v in ut32.items()},
            "source": "each SM unit's busy time per point from the committed capture (profiles/pipes.json), "
                      "x points, at the sampled SM clock; frac = the busiest unit's time over the kernel's"}
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms64,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 (positions, contraction and continuation rules in float-float; FP64 results)",
        "data": "synthetic: seeded LHAPDF-shaped grid and log-uniform queries (no real PDF set in the container)",
        "config": {"workload": WORKLOAD, "points_per_rank": n, "evals_per_step_per_rank": evals_step,
                   "class_counts": counts, "l2": "inputs + outputs 1.3 GB per step > 129 MB L2, no flush",
                   "parallelism": f"{world} independent replicas (weak scaling, no collective)"},
        "roofline": dict(roofline, peak_measured_dfma_tflops=fp64_meas.value / 1e12),
        "gpu_launches": 2 * args.steps,  # per step: the near and the far k_xf64 launch (all flavours + alpha_s)
        "clocks": clk,
        "e2e": {"value": world * evals_step / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": 16 * n,
                "d2h_bytes_per_step": 8 * n * (nf + 1), "ms_per_step": e2e_s * 1e3,
                "call": "xfxq2_all_flavours_host (pinned host buffers, alpha_s included)",
                "host_link_d2h_gbs": link["d2h_gbs"], "host_link_h2d_gbs": link["h2d_gbs"],
                "link_probe": "best of 5 timed copies each way on the step's own pinned buffers, after a warm copy",
                "link_bound_ms": e2e_bound_s * 1e3, "frac_of_link_bound": e2e_bound_s / e2e_s, "numa": numa},
        "paths": {
            "fp32": {"value": world * evals_step / (ms32 * 1e-3), "ms_per_step": ms32, "kernel_ms": k32,
                     "roofline": roofline32},
            "single_pid_fp64": {"value": world * n / (ms_pid * 1e-3), "ms_per_step": ms_pid},
            "alphas_fp64": {"value": world * n / (ms_as * 1e-3), "ms_per_step": ms_as},
            "mc_event_fp64": {"value": world * MC_EVENTS * (2 * nf + 1) / (ms_mc * 1e-3), "ms_per_step": ms_mc,
                              "events": MC_EVENTS},
            "mc_event_fp32": {"value": world * MC_EVENTS * (2 * nf + 1) / (ms_mc32 * 1e-3),
                              "ms_per_step": ms_mc32, "events": MC_EVENTS},
            "surrogate_bf16": surrogate,
            "surrogate_bf16_envelope_target": surrogate_env,
            "members_table2": members,
            "mc_integrate_fp64": mc_int,
            "single_subgrid_1e4": small,
            "adjoint_fp64": {"value": world * ADJ_POINTS * nf / (ms_adj * 1e-3), "ms_per_step": ms_adj,
                             "points": ADJ_POINTS, "unit": "(point, flavour) gradients/s",
                             "outputs": "d/dx, d/dQ^2 per point and d/d(knot values), FP64 atomics"},
        },
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sync()
        cpu, acc = cpu_baseline_leg(g, x, q2, out.cpu().numpy(), aout.cpu().numpy(), x32, q32,
                                    out32.cpu().numpy().astype(np.float64))
        line["cpu_baseline"] = cpu
        line["accuracy"] = acc
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--points", type=int, default=N_POINTS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-members", action="store_true")
    ap.add_argument("--only", choices=["fp64", "fp32", "surrogate", "adjoint"], default=None,
                    help="run only that path's step (a small case for profiling); prints its timing")
    ap.add_argument("--target", default="residual", choices=["residual", "envelope", "asinh"],
                    help="with --only surrogate: the surrogate's target")
    ap.add_argument("--law", default="bench", choices=["bench", "in", "lowx", "highq", "lowq", "lowx_highq",
                                                       "lowx_lowq"],
                    help="with --only fp64/fp32/adjoint: the benchmark's query law, or points of one class only")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
