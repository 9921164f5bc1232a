"""Benchmark: Monte Carlo radiative transfer on a hierarchical grid, 1 GB300.

Workload (default): the molecular-cloud model -- 256^3 root grid, lognormal
density (sigma_ln = 1.5) from a seeded k^-4 Gaussian random field, refined 3
levels by 2x2x2 where density exceeds 4^level x mean; isotropic external
field at 20 wavelengths (0.1-1000 um), kappa ~ lambda^-1.8, HG g = 0.5;
1e7 packages per wavelength; peel-off images 256x256 toward 6 observers;
FP32 tracing with FP64 accumulators.  One step = absorbed-energy trace with
peel-off (rt_peel) + dust-temperature solve (rt_dust_temperature).

Metric: cell crossings/s (trace + peel-off segments) and packages/s.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell crossings/s & packets/s on 1 GB300 vs roofline; p50/p99 job latency"
UNIT = "cell crossings/s"
# algorithmic bytes per unit of tracer work, as the method moves them: a
# trace crossing reads the leaf's density (4 B) and child word (4 B) and
# updates its FP64 accumulator (16 B read-modify-write); a peel-off crossing
# reads density and child word; an image deposit updates an FP64 pixel
BYTES_TRACE_CROSS = 4 + 4 + 16
BYTES_PEEL_CROSS = 4 + 4
BYTES_IMAGE_DEPOSIT = 16
# the same with the packed node word of this implementation (density or
# child index in one 32-bit word: one 4-byte read per visit)
BYTES_TRACE_CROSS_PACKED = 4 + 16
BYTES_PEEL_CROSS_PACKED = 4
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per crossing of
# the tracer (all its launches in a step: the emission round and the tiled
# rounds) and of the deferred peel-off kernel, from an ncu capture of every
# launch of one step of the same cloud at 128^3 root cells (tiles of 64^3,
# 1e6 packages per wavelength: 11.33 GB for 2.704e9 trace crossings, 1.206 GB
# for 1.809e9 peel-off crossings).  The bench line scales them by its own
# crossings on the default 256^3 workload (None whenever a kernel changes
# until it is captured again).  The tracer's figure is an upper bound there:
# the 128^3 case crosses tile faces twice as often per cell crossing.
# node descents per step of the default 256^3 cloud (a global read of an
# interior cell's child word each: 4 B in the roofline unit), counted with a
# build compiled with RT_COUNT_DESCENTS=1 (rt_descent_counts; the package
# histories are deterministic, so every run of this workload makes as many:
# its crossings matched the normal build's to the crossing)
BYTES_DESCENT = 4
DESCENTS_TRACE_DEFAULT = 3004187455
DESCENTS_PEEL_DEFAULT = 5202007659
NCU_TRACE_BYTES_PER_CROSSING = 11.329e9 / 2.704457093e9
NCU_PEEL_BYTES_PER_CROSSING = 1.206e9 / 1.808753762e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="cloud",
                    choices=["cloud", "disc", "batch", "serve", "peeltab", "split", "merge", "poly"],
                    help="cloud: the headline workload; disc/batch/serve: the other model families; "
                         "peeltab: accelerated against exact peel-off")
    ap.add_argument("--iters", type=int, default=30, help="disc: Lambda-iteration cap")
    ap.add_argument("--disc-packets", type=int, default=100_000_000)
    ap.add_argument("--disc-min-hits", type=float, default=1000.0,
                    help="disc: cells with fewer deposits are left out of the stop rule")
    ap.add_argument("--sub-level", type=int, default=-1,
                    help="disc: compare full Lambda iterations with subiterations below this level")
    ap.add_argument("--ali", action="store_true", help="disc subiterations: also 30 full ALI steps")
    ap.add_argument("--ali-max-lambda", type=float, nargs="+", default=[0.999],
                    help="disc ALI: cap of Lambda_b (one run per value, with the first --ali-min)")
    ap.add_argument("--ali-min", type=int, nargs="+", default=[100],
                    help="disc ALI: minimum packages a cell sends for its diagonal operator (one run per value)")
    ap.add_argument("--split-runs", type=int, default=20, help="split: runs with and without resampling")
    ap.add_argument("--split-packets", type=int, default=2_000_000, help="split: initial packages per run")
    ap.add_argument("--split-lambda", type=float, default=4.0, help="split: wavelength (um) of the field")
    ap.add_argument("--merge-packets", type=int, default=20_000_000, help="merge: packages per wavelength")
    ap.add_argument("--poly-group", type=int, default=4, help="poly: bins per polychromatic package")
    ap.add_argument("--poly-packets", type=int, default=1_000_000, help="poly: packages per bin / per group")
    ap.add_argument("--flux-frac", type=float, default=0.05,
                    help="disc subiterations: full step once the emission below the level changed by this fraction")
    ap.add_argument("--models", type=int, default=64, help="batch: models per launch")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="serve: seconds of Poisson arrivals")
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-max-packets", type=float, default=1e8)
    ap.add_argument("--serve-slots", type=int, default=2)
    ap.add_argument("--serve-batch", type=int, default=64)
    ap.add_argument("--serve-batch-packets", type=float, default=1e7,
                    help="serve: a launch takes jobs while their packages sum to at most this (0: no limit)")
    ap.add_argument("--line-serve-seconds", type=float, default=15.0,
                    help="seconds of Poisson arrivals for the serving figures of the default line (0: none)")
    ap.add_argument("--n-root", type=int, default=256)
    ap.add_argument("--levels", type=int, default=3)
    ap.add_argument("--threshold-scale", type=float, default=1.0,
                    help="cloud: refine where density > c x 4^l x mean (0.067: 8%% of the equivalent uniform cells)")
    ap.add_argument("--n-lambda", type=int, default=20)
    ap.add_argument("--packets-per-bin", type=int, default=10_000_000)
    ap.add_argument("--n-pix", type=int, default=256)
    ap.add_argument("--precision", type=int, default=32)
    ap.add_argument("--cpu-packets-per-bin", type=int, default=0, help="oracle sample size (0: auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--rr-wmin", type=float, default=1e-4, help="Russian roulette below this fraction of W0")
    ap.add_argument("--rr-p", type=float, default=0.9)
    ap.add_argument("--block-size", type=int, default=0)
    ap.add_argument("--refill", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--tiles", type=int, default=-1,
                    help="tiled tracing: tile edge in root cells (power of two), 0 off, -1 automatic")
    ap.add_argument("--peel-queue", type=int, default=-1,
                    help="deferred peel-off queue in records, 0 inline, -1 default")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

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
        if self.t:
            self.t.join(timeout=2)
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
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def l2_read_gbs(ctx, dev):
    """L2 read bandwidth measured here by the library's diagnostic kernel:
    16-byte L2-only loads over a zeroed 48 MB buffer, 40 passes a launch."""
    import torch

    from paper_1206_3710_gb300 import rt
    buf = torch.zeros(48 * 2 ** 20 // 8, dtype=torch.float64, device=dev)
    return rt.rt_l2_read_bandwidth(ctx, buf, reps=40)


def make_model(a):
    from paper_1206_3710_gb300 import synth
    return synth.cloud(n_root=a.n_root, levels=a.levels, n_lambda=a.n_lambda, packets_per_bin=a.packets_per_bin,
                       n_pix=a.n_pix, threshold_scale=a.threshold_scale)


def workload_config(a, m):
    thr = "4^l x mean" if a.threshold_scale == 1.0 else f"{a.threshold_scale:g} x 4^l x mean"
    uniform = m.tree.n_cells / float(a.n_root << a.levels) ** 3
    return {"workload": f"molecular cloud: {a.n_root}^3 root, {a.levels} levels (threshold {thr}), "
                        f"lognormal sigma_ln=1.5, {a.n_lambda} wavelengths, external isotropic field, "
                        f"{a.packets_per_bin:.0e} packages/wavelength, peel-off {m.observers.n_obs}x"
                        f"{a.n_pix}^2, FP32 trace + FP64 accumulators",
            "n_cells": int(m.tree.n_cells), "n_levels": int(m.tree.n_levels),
            "fraction_of_uniform_cells": uniform,
            "packets_per_step": int(a.packets_per_bin * a.n_lambda * len(m.sources)),
            "l2_policy": "inputs larger than L2 (grid + per-wavelength FP64 absorbed arrays)"}


def dust_arrays(m):
    kabs = (1 - m.optics.albedo) * m.optics.kappa_ext
    return m.optics.lambda_um, kabs, m.optics.dnu


def oracle_sample_size(a, m, tree, cores, want_seconds=12.0):
    """Packages per wavelength for which one oracle trace of the workload on
    `cores` threads takes about want_seconds (grown from a small probe)."""
    import oracle
    ppb = 50
    while True:
        t1 = time.perf_counter()
        oracle.trace(tree, m.sources, m.optics, ppb, seed=1002, observers=m.observers, n_threads=cores,
                     rr_wmin=a.rr_wmin, rr_p=a.rr_p)
        dt = time.perf_counter() - t1
        if dt > 0.2 * want_seconds or ppb >= a.packets_per_bin:
            break
        ppb = int(ppb * min(8.0, max(2.0, 0.5 * want_seconds / max(dt, 1e-3))))
    return max(1, min(a.packets_per_bin, int(ppb * want_seconds / max(dt, 1e-3))))


def _oracle_rate(a, m, tree, ppb, cores, seed=1002, iter_=0):
    import oracle
    t1 = time.perf_counter()
    r = oracle.trace(tree, m.sources, m.optics, ppb, seed=seed, iter_=iter_, observers=m.observers,
                     n_threads=cores, rr_wmin=a.rr_wmin, rr_p=a.rr_p)
    dt = time.perf_counter() - t1
    L = r["ledger"]
    return L["n_cross"] + L["n_peel_cross"], L["n_packets"], dt


def cpu_baseline(a, m, packets_per_bin=None):
    """Time the FP64 oracle (as it stands) on a bounded sample of the
    workload: all host cores, and one core on a smaller sample."""
    import oracle
    t0 = time.perf_counter()
    tree = oracle.Tree(m.tree)
    t_build = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    ppb = packets_per_bin or oracle_sample_size(a, m, tree, cores)
    cross, npk, dt = _oracle_rate(a, m, tree, ppb, cores)
    ppb1 = max(1, ppb // (2 * cores))
    cross1, npk1, dt1 = _oracle_rate(a, m, tree, ppb1, 1)
    return {"value": cross / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "packets_per_s": npk / dt,
            "sample": f"{ppb} packages per wavelength x {a.n_lambda} wavelengths on the full grid with "
                      f"{m.observers.n_obs} peel-off observers ({int(npk)} packages, "
                      f"{int(cross)} crossings, {dt:.2f} s; tree build {t_build:.1f} s excluded)",
            "single_thread": {"value": cross1 / dt1, "unit": UNIT, "cores": 1, "packets_per_s": npk1 / dt1,
                              "sample": f"{ppb1} packages per wavelength ({int(npk1)} packages, {dt1:.2f} s)"}}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    m = make_model(a)
    import oracle
    tree = oracle.Tree(m.tree)
    cores = os.cpu_count() or 1
    # the same sample size as the cpu_baseline leg of the GPU arm: one step
    # is about 12 s of oracle work on all host cores
    ppb = a.cpu_packets_per_bin or oracle_sample_size(a, m, tree, cores)
    for _ in range(a.warmup):
        _oracle_rate(a, m, tree, max(1, ppb // 10), cores)
    tot_cross, tot_pk, t = 0.0, 0.0, 0.0
    for s in range(a.steps):
        c, p, dt = _oracle_rate(a, m, tree, ppb, cores, iter_=s)
        t += dt
        tot_cross += c
        tot_pk += p
    v = tot_cross / t
    sample = f"{ppb} packages per wavelength x {a.n_lambda} wavelengths per step, full grid, peel-off"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * t / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded lognormal cloud)",
            "config": workload_config(a, m), "packets_per_s": tot_pk / t,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def shard_params(rank: int, packets_per_bin: int) -> dict:
    """Rank r traces packages [r*n, (r+1)*n) of every (source, bin): one Philox
    key for all ranks and disjoint package indices, so the ranks together are
    one run of world*n packages per bin (each rank's weights carry the full
    source energy: their mean is that run's result)."""
    return dict(job=0, packet_offset=rank * packets_per_bin)


def combine_shards(dist, world: int, *fields):
    """The one exchange step of a sharded run (Sect. 5.2: results combine
    only at the end): every rank's FP64 fields (absorbed energy, images)
    become the mean over the ranks, i.e. the single run of world*n packages
    per bin, on every rank (the temperature solve and the next Lambda step
    need the combined field)."""
    if world <= 1:
        return
    for f in fields:
        dist.all_reduce(f)
        f.mul_(1.0 / world)


def reduce_over_ranks(dist, t_ms: float, counts, device):
    """Max of the ranks' timed spans and sums of their work counters."""
    import torch
    tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ct = torch.tensor([float(c) for c in counts], dtype=torch.float64, device=device)
    dist.all_reduce(ct)
    return float(tt.item()), [float(v) for v in ct.tolist()]


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    if a.workload != "cloud":
        import bench_families
        bench_families.run(a)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_1206_3710_gb300 import rt
    t_gen = time.perf_counter()
    m = make_model(a)
    t_gen = time.perf_counter() - t_gen
    ctx = rt.Context(local)
    ctx.set_tiles(a.tiles)
    ctx.set_peel_queue(a.peel_queue)
    grid = rt.Grid(ctx, m.tree)
    nl = m.optics.n_lambda
    nc = grid.n_cells
    obs = m.observers
    absorbed = torch.zeros((nl, nc), dtype=torch.float64, device=dev)
    images = torch.zeros((obs.n_obs, nl, obs.ny, obs.nx), dtype=torch.float64, device=dev)
    T = torch.zeros(nc, dtype=torch.float64, device=dev)
    lam, kabs, dnu = dust_arrays(m)
    stream = torch.cuda.current_stream(dev)
    kw = dict(seed=1002, precision=a.precision, packets_per_bin=a.packets_per_bin,
              rr_wmin=a.rr_wmin, rr_p=a.rr_p,
              block_size=a.block_size, refill_threshold=a.refill, blocks_per_sm=a.blocks_per_sm,
              **shard_params(rank, a.packets_per_bin))

    def step():
        absorbed.zero_()
        images.zero_()
        led = rt.rt_peel(ctx, grid, m.sources, m.optics, obs, images, absorbed, stream=stream, **kw)
        combine_shards(dist, world, absorbed, images)
        rt.rt_dust_temperature(ctx, grid, absorbed, nl, lam, kabs, dnu, T, stream=stream)
        return led

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0.record(stream)
    leds = [step() for _ in range(a.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_ms = ev0.elapsed_time(ev1)
    cross = sum(L["n_cross"] + L["n_peel_cross"] for L in leds)
    pk = sum(L["n_packets"] for L in leds)
    if world > 1:
        t_ms, (cross, pk) = reduce_over_ranks(dist, t_ms, [cross, pk], dev)
    value = cross / (t_ms * 1e-3)

    # rooflines of the tracer and of the deferred peel-off kernel (device time
    # of each launch from the library's events on the launching stream)
    L0 = leds[-1]
    kern_ms = statistics.mean(L["kernel_ms"] for L in leds)
    peel_ms = statistics.mean(L["peel_ms"] for L in leds)
    deposits = L0["n_scatter"] * obs.n_obs - L0["n_peel_out"]
    peak, peak_kind = peaks()
    l2_peak = l2_read_gbs(ctx, dev)
    trace_bytes = BYTES_TRACE_CROSS * L0["n_cross"]
    peel_bytes = BYTES_PEEL_CROSS * L0["n_peel_cross"] + BYTES_IMAGE_DEPOSIT * deposits
    trace_packed = BYTES_TRACE_CROSS_PACKED * L0["n_cross"]
    peel_packed = BYTES_PEEL_CROSS_PACKED * L0["n_peel_cross"] + BYTES_IMAGE_DEPOSIT * deposits
    if L0["n_peel_deferred"] < L0["n_scatter"]:  # some peel-offs ran inline in the tracer
        trace_bytes, peel_bytes = trace_bytes + peel_bytes, 0
        trace_packed, peel_packed = trace_packed + peel_packed, 0
    default_cloud = ((a.n_root, a.levels, a.threshold_scale, a.n_lambda, a.packets_per_bin, a.precision)
                     == (256, 3, 1.0, 20, 10_000_000, 32) and world == 1
                     and L0["n_peel_deferred"] == L0["n_scatter"])
    descents = (DESCENTS_TRACE_DEFAULT, DESCENTS_PEEL_DEFAULT) if default_cloud else (None, None)
    if default_cloud:  # the descent term of the unit, counted once for this workload
        trace_bytes += BYTES_DESCENT * DESCENTS_TRACE_DEFAULT
        trace_packed += BYTES_DESCENT * DESCENTS_TRACE_DEFAULT
        peel_bytes += BYTES_DESCENT * DESCENTS_PEEL_DEFAULT
        peel_packed += BYTES_DESCENT * DESCENTS_PEEL_DEFAULT
    achieved = trace_bytes / (kern_ms * 1e-3) / 1e9
    trace_traffic = peel_traffic = None
    if default_cloud and NCU_TRACE_BYTES_PER_CROSSING is not None:
        trace_traffic = NCU_TRACE_BYTES_PER_CROSSING * L0["n_cross"]
    if default_cloud and NCU_PEEL_BYTES_PER_CROSSING is not None:
        peel_traffic = NCU_PEEL_BYTES_PER_CROSSING * L0["n_peel_cross"]
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": trace_traffic,
            "traffic_basis": "per step: ncu DRAM bytes per crossing of a 128^3 step, times this step's crossings",
            "peak_kind": peak_kind, "kernel": "trace_kernel<float,1,0,0>",
            "kernel_ms": kern_ms, "alg_bytes_per_launch": trace_bytes,
            "bytes_per_unit": {"trace_crossing": BYTES_TRACE_CROSS, "peel_crossing": BYTES_PEEL_CROSS,
                               "image_deposit": BYTES_IMAGE_DEPOSIT, "descent": BYTES_DESCENT},
            "descents_per_step": {"trace": descents[0], "peel": descents[1]},
            "packed_node_word": {"bytes_per_trace_crossing": BYTES_TRACE_CROSS_PACKED,
                                 "frac": trace_packed / (kern_ms * 1e-3) / 1e9 / peak},
            # the tiled rounds keep each round's cells in L2: the same bytes
            # against the L2 read bandwidth measured in this run
            "l2": {"peak": l2_peak, "unit": "GB/s", "frac": achieved / l2_peak,
                   "peak_kind": "measured (rt_l2_read_bandwidth: L2-only 16-byte loads over a 48 MB buffer)"}}
    peel_roof = None
    if peel_ms > 0:
        pa = peel_bytes / (peel_ms * 1e-3) / 1e9
        peel_roof = {"kernel": "peel_kernel<float>", "bound": "hbm", "achieved": pa, "peak": peak, "unit": "GB/s",
                     "frac": pa / peak, "kernel_ms": peel_ms, "alg_bytes_per_launch": peel_bytes,
                     "traffic": peel_traffic,
                     "crossings_per_s": L0["n_peel_cross"] / (peel_ms * 1e-3),
                     "packed_node_word": {"frac": peel_packed / (peel_ms * 1e-3) / 1e9 / peak},
                     "l2": {"peak": l2_peak, "frac": pa / l2_peak}}

    out = None
    if rank == 0:
        e2e = None
        if not a.no_e2e:
            e2e = e2e_run(a, m, ctx, dev, stream, kw, lam, kabs, dnu)
        cpu = None
        if not a.no_cpu_baseline and world == 1:
            cpu = cpu_baseline(a, m, a.cpu_packets_per_bin or None)
        serving = None
        if a.line_serve_seconds > 0 and world == 1:
            serving = serving_figures(a, ctx, dev)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": t_ms / a.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32" if a.precision == 32 else "f64",
               "data": "synthetic (seeded lognormal cloud, random-field density)",
               "config": workload_config(a, m), "packets_per_s": pk / (t_ms * 1e-3),
               "crossings_per_step": {"trace": L0["n_cross"], "peel": L0["n_peel_cross"]},
               "scatterings_per_step": L0["n_scatter"], "roofline": roof, "roofline_peel_kernel": peel_roof,
               "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "serving": serving,
               "gpu_launches": sum(int(L["n_launches"]) + 2 for L in leds),  # + dust table and temperature
               "tiling": {"tiles": L0["n_tiles"], "rounds_per_step": L0["n_rounds"]},
               "energy_balance": (L0["emitted"] - L0["absorbed"] - L0["escaped"]) / L0["emitted"],
               "model_generation_s": t_gen}
        print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def serving_figures(a, ctx, dev):
    """The serving pattern on a bounded stream: Poisson arrivals of jobs drawn
    from the cloud, disc, clump and batch model families (1e5..1e8 packages,
    1..30 wavelengths), p50/p99 latency, packages/s served, the same jobs one
    at a time, and all of them submitted at once."""
    import torch

    import bench_families
    from paper_1206_3710_gb300 import rt, synth
    res = bench_families.serve_measure(rt, synth, ctx, torch, a.line_serve_seconds, a.serve_rate,
                                       a.serve_max_packets, slots=a.serve_slots, max_batch_jobs=a.serve_batch,
                                       max_batch_packets=a.serve_batch_packets)
    res.pop("library", None)
    # the same pattern with small jobs (1e5..1e6 packages), where one job
    # leaves most of the GPU idle and continuous batching pays
    small = bench_families.serve_measure(rt, synth, ctx, torch, a.line_serve_seconds, a.serve_rate, 1e6,
                                         slots=a.serve_slots, max_batch_jobs=a.serve_batch,
                                         max_batch_packets=a.serve_batch_packets)
    res["small_jobs"] = {k: small[k] for k in ("jobs", "packets_per_job", "p50_ms", "p99_ms", "served_packets_per_s",
                                               "burst_packets_per_s", "serial_packets_per_s", "burst_over_serial")}
    return res


def e2e_run(a, m, ctx, dev, stream, kw, lam, kabs, dnu):
    """Same metric through the public API with host buffers.  The mesh is
    uploaded once (rt_build_grid, before the timed region); every step then
    uploads the density from pinned host memory (rt_grid_set_density), traces
    (rt_peel), solves the temperatures (rt_dust_temperature) and copies the
    step's results, the dust temperatures and the peel-off images (Sects.
    4.1-4.2), to pinned host memory; the absorbed energy per bin stays on the
    device, as between the steps of a Lambda iteration.  A step's copies run
    on a second stream while the next step traces (two sets of device and
    host outputs); one untimed step first."""
    import torch

    from paper_1206_3710_gb300 import rt
    obs = m.observers
    nl = m.optics.n_lambda
    nc = m.tree.n_cells
    dens = torch.empty(nc, dtype=torch.float64, pin_memory=True)
    dens.numpy()[:] = m.tree.density
    grid = rt.Grid(ctx, m.tree)
    comp = torch.cuda.Stream(dev)
    copy = torch.cuda.Stream(dev)
    bufs = []
    for _ in range(2):
        shapes = ((nl, nc), (obs.n_obs, nl, obs.ny, obs.nx), (nc,))
        bufs.append({"dev": [torch.empty(sh, dtype=torch.float64, device=dev) for sh in shapes],
                     "host": [torch.empty(sh, dtype=torch.float64, pin_memory=True) for sh in shapes[1:]],
                     "done": torch.cuda.Event(), "copied": torch.cuda.Event()})
    steps = max(1, a.steps)
    cross = 0
    t0 = 0.0
    for i in range(steps + 1):
        if i == 1:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        b = bufs[i % 2]
        ab, im, T = b["dev"]
        comp.wait_event(b["copied"])          # this set's copies of two steps ago are done
        grid.set_density(dens.numpy(), stream=comp)
        with torch.cuda.stream(comp):
            ab.zero_()
            im.zero_()
        led = rt.rt_peel(ctx, grid, m.sources, m.optics, obs, im, ab, stream=comp, **kw)
        rt.rt_dust_temperature(ctx, grid, ab, nl, lam, kabs, dnu, T, stream=comp)
        b["done"].record(comp)
        copy.wait_event(b["done"])
        with torch.cuda.stream(copy):
            for h, d in zip(b["host"], b["dev"][1:]):    # images, temperatures
                h.copy_(d, non_blocking=True)
        b["copied"].record(copy)
        if i >= 1:
            cross += led["n_cross"] + led["n_peel_cross"]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    grid.close()
    h2d = dens.numel() * 8
    d2h = sum(h.numel() * 8 for h in bufs[0]["host"])
    return {"value": cross / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": steps, "ms_per_step": 1e3 * dt / steps,
            "pattern": "mesh uploaded once; per step: density up from pinned memory, trace, temperatures, "
                       "temperatures and images down to pinned memory overlapped with the next step"}

if __name__ == "__main__":
    main()
