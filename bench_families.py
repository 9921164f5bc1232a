"""Measurements of the other model families (bench.py --workload disc|batch|serve).

* disc  -- circumstellar disc (64^3 root, <=10 levels, ~9e6 cells), 30
           wavelengths, 1e8 packages per trace, Lambda iteration of the dust
           temperature until max dT/T < 1e-3 (cells with >= 1e3 deposits) or
           30 iterations (Sect. 4.2, Eq. 2).
* batch -- 64 models (roots 32^3/64^3/128^3, 0-4 levels, clump or lognormal,
           16 wavelengths, 1e5-1e7 packages) in one autotuned, graph-captured
           FP32 launch, against one plain FP64 launch per model.
* serve -- Poisson arrivals of jobs drawn from the model families; the job
           server admits by device-memory footprint and batches continuously;
           p50/p99 latency and packages/s against running the same jobs one
           at a time.
* peeltab -- accelerated peel-off (Sect. 2.4) against exact peel-off
           marches on the molecular cloud (6 axis observers) and the disc
           (5 observers 2 degrees above the plane): table build time, peel-off
           kernel time, crossings, image relative RMS difference.
* merge -- Sect. 4.1: a full-resolution lognormal cloud cube (256^3) against
           the hierarchical model built from it (32^3 root, 3 levels, cells
           combined while tau_V <= 0.05 and contrast < 30): cells, trace and
           peel-off time, and the relative mean and RMS differences of the
           scattered-light maps (Eqs. 6-7).
* poly -- polychromatic packages (groups of 4 bins) against monochromatic
           ones on a 128^3 molecular cloud (20 wavelengths, external field,
           6 observers): time per run, per-bin noise of the absorbed energy
           and of the images (two seeds), and the efficiency ratio
           t_mono noise_mono^2 / (t_poly noise_poly^2).
* split -- resampling at grid boundaries (Sect. 2.3, Table 1): the 4 um
           radiation field of the molecular cloud from the external field and
           from embedded point sources, R runs with and without splitting
           (factor 4) from the same number of initial packages; RMS deviation
           per hierarchy level from the mean of all runs, and trace time.
Each prints one JSON line.
"""
from __future__ import annotations

import json
import math
import threading
import time

import numpy as np


def _clock_start(local=0):
    from bench import ClockSampler
    c = ClockSampler(local)
    c.start()
    return c


def run(a):
    import torch
    from paper_1206_3710_gb300 import rt, synth
    torch.cuda.set_device(0)
    ctx = rt.Context(0)
    {"disc": run_disc, "batch": run_batch, "serve": run_serve, "peeltab": run_peeltab,
     "split": run_split, "merge": run_merge, "poly": run_poly}[a.workload](a, rt, synth, ctx, torch)


def run_disc_subiter(a, rt, synth, ctx, torch):
    """Sect. 4.2's comparison: the same number of steps of full Lambda
    iterations and of automatically chosen subiterations (App. B) on the disc;
    wall time, step kinds and the temperature difference between the two."""
    m = synth.disc(packets=a.disc_packets)
    g = rt.Grid(ctx, m.tree)
    kw = dict(seed=1003, precision=32, packets_total=a.disc_packets, rr_wmin=1e-4, rr_p=0.9,
              dust_packets_total=a.disc_packets, min_hits=1000, tol=0.0)
    leaf = m.tree.refine_flags == 0
    h = m.tree.box[0] / m.tree.root[0] * 0.5 ** synth_levels(m.tree)
    mass = m.tree.density * h ** 3
    T_full = torch.zeros(g.n_cells, dtype=torch.float64, device="cuda")
    clk = _clock_start()
    rf = rt.rt_lambda_subiterate(ctx, g, m.sources, m.optics, T_full, sub_level=a.sub_level,
                                 schedule=["full"] * a.iters, **kw)
    T_sub = torch.zeros_like(T_full)
    rs = rt.rt_lambda_subiterate(ctx, g, m.sources, m.optics, T_sub, sub_level=a.sub_level, max_iter=a.iters,
                                 select_frac=0.25, flux_frac=a.flux_frac, **kw)
    ali = None
    if a.ali:
        ali = []
        runs = [(amin, a.ali_max_lambda[0]) for amin in a.ali_min] + \
            [(a.ali_min[0], cap) for cap in a.ali_max_lambda[1:]]
        for amin, cap in runs:
            T_ali = torch.zeros_like(T_full)
            ra = rt.rt_lambda_subiterate(ctx, g, m.sources, m.optics, T_ali, sub_level=a.sub_level,
                                         schedule=["full"] * a.iters, ali=True, ali_min_packages=amin,
                                         ali_max_lambda=cap, **kw)
            ta = T_ali.cpu().numpy()[leaf]
            tfa = T_full.cpu().numpy()[leaf]
            lv = synth_levels(m.tree)[leaf]
            per_level = [[int(l), int((lv == l).sum()), round(float(tfa[lv == l].mean()), 2),
                          round(float(ta[lv == l].mean()), 2)] for l in range(int(lv.max()) + 1) if (lv == l).any()]
            ali.append({"ali_min_packages": amin, "ali_max_lambda": cap, "ms": ra["ms"], "history": ra["history"],
                        "mean_T_K": float(ta.mean()), "mean_T_full_K": float(tfa.mean()),
                        "mass_weighted_mean_dT_vs_full_K": float(np.sum(mass[leaf] * (ta - tfa)) / mass[leaf].sum()),
                        "per_level_leaves_meanT_full_ali": per_level,
                        # mass-weighted mean |absorbed - emitted| per unit mass after the last step
                        "imbalance_last_ali": ra["imbalance"][-1], "imbalance_last_full": rf["imbalance"][-1]})
    clocks = clk.stop()
    tf, ts = T_full.cpu().numpy()[leaf], T_sub.cpu().numpy()[leaf]
    w = mass[leaf]
    d = ts - tf
    line = {"metric": "Lambda iteration: full steps against subiterations (App. B), same number of steps",
            "workload": "disc_subiter", "n_cells": int(m.tree.n_cells), "sub_level": a.sub_level,
            "flux_frac": a.flux_frac,
            "steps": a.iters, "full_ms": rf["ms"], "subiter_ms": rs["ms"], "speedup": rf["ms"] / rs["ms"],
            "subiter_steps": rs["steps"], "subiter_step_ms": rs["step_ms"], "full_step_ms": rf["step_ms"],
            "imbalance": rs["imbalance"],
            "rms_dT_K": float(np.sqrt(np.mean(d * d))), "mass_weighted_rms_dT_K": float(np.sqrt(np.sum(w * d * d) / w.sum())),
            "rms_T_K": float(np.sqrt(np.mean(tf * tf))), "mean_dT_K": float(d.mean()),
            "history_full": rf["history"], "history_subiter": rs["history"], "ali_full_steps": ali,
            "clocks": clocks}
    print(json.dumps(line))


def synth_levels(tree):
    """Level of every cell of a level-ordered tree description."""
    n0 = int(np.prod(tree.root))
    lev = np.zeros(tree.n_cells, np.int64)
    off, cnt = n0, n0
    for l in range(len(tree.n_refined) - 1):
        nxt = 8 * int(tree.n_refined[l])
        lev[off:off + nxt] = l + 1
        off += nxt
    return lev


def run_disc(a, rt, synth, ctx, torch):
    if a.sub_level >= 0:
        return run_disc_subiter(a, rt, synth, ctx, torch)
    t0 = time.perf_counter()
    m = synth.disc(packets=a.disc_packets)
    t_gen = time.perf_counter() - t0
    g = rt.Grid(ctx, m.tree)
    T = torch.zeros(g.n_cells, dtype=torch.float64, device="cuda")
    kw = dict(seed=1003, precision=32, packets_total=a.disc_packets, rr_wmin=1e-4, rr_p=0.9)
    clk = _clock_start()
    res = rt.rt_lambda_iterate(ctx, g, m.sources, m.optics, T, max_iter=a.iters, tol=1e-3, min_hits=a.disc_min_hits,
                               dust_packets_total=a.disc_packets, **kw)
    clocks = clk.stop()
    src, dust = res["source_ledger"], res["dust_ledger"]
    Tn = T.cpu().numpy()
    leaf = m.tree.refine_flags == 0
    line = {"metric": "Lambda iteration: cell crossings/s and iterations to max dT/T < 1e-3",
            "workload": "disc", "n_cells": int(m.tree.n_cells), "n_levels": int(m.tree.n_levels),
            "tau_cell_threshold": m.tau_cell_thr, "iterations": res["n_iter"], "history": res["history"],
            "packages_per_trace": a.disc_packets, "min_hits": a.disc_min_hits,
            "total_ms": res["ms"], "ms_per_iteration": res["ms"] / max(1, res["n_iter"] + 1),
            "source_trace": {k: src[k] for k in ("n_packets", "n_cross", "n_scatter", "kernel_ms")},
            "dust_trace_last": {k: dust[k] for k in ("n_packets", "n_cross", "n_scatter", "kernel_ms")},
            "dust_cross_per_s": dust["n_cross"] / (dust["kernel_ms"] * 1e-3) if dust["kernel_ms"] else None,
            "T_leaf_min_median_max": [float(Tn[leaf].min()), float(np.median(Tn[leaf])), float(Tn[leaf].max())],
            "model_generation_s": t_gen, "clocks": clocks, "dtype": "f32 trace, f64 accumulators and solve"}
    print(json.dumps(line))


def _batch_jobs(rt, ctx, torch, models, precision):
    grids, jobs = [], []
    for i, m in enumerate(models):
        g = rt.Grid(ctx, m.tree)
        grids.append(g)
        ab = torch.zeros((m.optics.n_lambda, g.n_cells), dtype=torch.float64, device="cuda")
        jobs.append(rt.Job(g, m.sources, m.optics, ab, seed=m.seed, job=i, precision=precision,
                           packets_per_bin=m.packets_per_bin, rr_wmin=1e-4, rr_p=0.9))
    return grids, jobs


def run_batch(a, rt, synth, ctx, torch):
    t0 = time.perf_counter()
    models = synth.batch_models(n_models=a.models, seed=1004)
    t_gen = time.perf_counter() - t0
    grids, jobs32 = _batch_jobs(rt, ctx, torch, models, 32)
    tune = rt.rt_autotune(ctx, jobs32, sample_fraction=0.05)
    batch = rt.Batch(ctx, jobs32)
    for _ in range(max(1, a.warmup)):
        batch.run()
    torch.cuda.synchronize()
    clk = _clock_start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    leds = None
    for _ in range(a.steps):
        leds = batch.run()
    ev1.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms_batch = ev0.elapsed_time(ev1) / a.steps
    pk = sum(x["n_packets"] for x in leds)
    cross = sum(x["n_cross"] for x in leds)
    res32 = [j.absorbed.sum().item() for j in jobs32]
    # plain FP64 launches, one per model
    _, jobs64 = _batch_jobs(rt, ctx, torch, models, 64)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    leds64 = []
    for j in jobs64:
        leds64.append(rt.rt_trace(ctx, j.grid, j.sources, j.optics, j.absorbed, **j.params))
    torch.cuda.synchronize()
    ms_plain = (time.perf_counter() - t1) * 1e3
    res64 = [j.absorbed.sum().item() for j in jobs64]
    rel = [abs(x / y - 1) for x, y in zip(res32, res64) if y > 0]
    line = {"metric": "batched FP32 packets/s vs one plain FP64 launch per model",
            "workload": "batch", "models": len(models), "packets_per_run": int(pk), "crossings_per_run": int(cross),
            "batched_fp32": {"ms": ms_batch, "packets_per_s": pk / (ms_batch * 1e-3),
                             "cross_per_s": cross / (ms_batch * 1e-3), "autotune": tune},
            "plain_fp64_per_model": {"ms": ms_plain, "packets_per_s": pk / (ms_plain * 1e-3)},
            "speedup": ms_plain / ms_batch,
            "accuracy": {"max_rel_diff_total_absorbed": max(rel), "median": float(np.median(rel))},
            "model_generation_s": t_gen, "clocks": clocks}
    print(json.dumps(line))


def _serve_library(synth):
    lib = [synth.tiny_clump(),
           synth.cloud(n_root=64, levels=3, n_lambda=30, seed=2101, packets_per_bin=0, n_pix=64),
           synth.cloud(n_root=128, levels=3, n_lambda=30, seed=2102, packets_per_bin=0, n_pix=64),
           synth.disc(n_root=32, max_level=7, n_lambda=30, packets=0, target_cells=3e5, max_cells=2_000_000)]
    lib += synth.batch_models(n_models=4, seed=2103, n_lambda=30, roots=(32, 64), max_levels=3)
    return lib


def _optics_subset(synth, m, nl, rng):
    """A job's wavelengths: nl bins of the model's grid (its dust law)."""
    idx = np.sort(rng.choice(m.optics.n_lambda, size=nl, replace=False))
    o = m.optics
    opt = synth.Optics(o.lambda_um[idx], o.kappa_ext[idx], o.albedo[idx], o.g_hg[idx], o.dnu[idx])
    src = []
    for s in m.sources:
        be = s.bin_energy[idx] if s.bin_energy is not None and len(s.bin_energy) == o.n_lambda else np.full(nl, 1.0 / nl)
        src.append(synth.Source(s.kind, bin_energy=be, pos=s.pos))
    return opt, src


def serve_jobs(synth, seconds, rate, max_packets, seed=1005):
    """A seeded Poisson stream of jobs drawn from the serving library's model
    families: (arrival time, model id, sources, optics, trace parameters)."""
    rng = np.random.default_rng(seed)
    library = _serve_library(synth)
    n_jobs = max(1, int(seconds * rate))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_jobs))
    jobs = []
    for i in range(n_jobs):
        mid = int(rng.integers(len(library)))
        m = library[mid]
        nl = int(rng.integers(1, min(30, m.optics.n_lambda) + 1))
        opt, src = _optics_subset(synth, m, nl, rng)
        total = math.exp(rng.uniform(math.log(1e5), math.log(max_packets)))
        ppb = max(1, int(total / nl))
        jobs.append((arrivals[i], mid, src, opt, dict(seed=5000 + i, job=i, precision=32, packets_per_bin=ppb,
                                                      rr_wmin=1e-4, rr_p=0.9, per_lambda=False)))
    return library, jobs


def serve_measure(rt, synth, ctx, torch, seconds, rate, max_packets, slots=2, max_batch_jobs=64,
                  batch_window_ms=1.0, max_batch_packets=1e7):
    """Serving under Poisson arrivals (latency p50/p99 from submission to the
    result being ready on the device, packages/s), the same jobs one at a
    time with their own launches, and the burst capacity (all jobs submitted
    at once).  Results stay on the device and are released, in all three."""
    library, jobs = serve_jobs(synth, seconds, rate, max_packets)
    n_jobs = len(jobs)
    arrivals = np.array([j[0] for j in jobs])
    free = torch.cuda.mem_get_info()[0]

    def server():
        srv = rt.Server(ctx, hbm_budget=int(0.5 * free), slots=slots, max_batch_jobs=max_batch_jobs,
                        batch_window_ms=batch_window_ms, max_batch_packets=int(max_batch_packets))
        for mid, m in enumerate(library):
            srv.add_model(mid, m.tree)
        # warm-up: the first job of each model makes its grid resident
        first = {}
        for (t_arr, mid, src, opt, prm) in jobs:
            first.setdefault(mid, (src, opt, prm))
        for mid, (src, opt, prm) in first.items():
            t = srv.submit(mid, src, opt, **dict(prm, packets_per_bin=100))
            srv.wait(t, 600)
            srv.release(t)
        return srv

    srv = server()
    tickets = [None] * n_jobs
    done_lat = [None] * n_jobs
    leds = [None] * n_jobs

    def collector():
        for i in range(n_jobs):
            while tickets[i] is None:
                time.sleep(0.0005)
            srv.wait(tickets[i], 3600)
            _, led, lat = srv.poll(tickets[i])
            srv.release(tickets[i])
            done_lat[i], leds[i] = lat, led

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    start = time.perf_counter()
    for i, (t_arr, mid, src, opt, prm) in enumerate(jobs):
        dt = start + t_arr - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets[i] = srv.submit(mid, src, opt, **prm)
    th.join()
    wall = time.perf_counter() - start
    srv.close()
    lat = np.array(done_lat)
    pk = sum(x["n_packets"] for x in leds)
    # the same jobs one at a time, each with its own launch (no overlap, no batching)
    grids = [rt.Grid(ctx, m.tree) for m in library]
    bufs = [torch.zeros((1, g.n_cells), dtype=torch.float64, device="cuda") for g in grids]
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for (t_arr, mid, src, opt, prm) in jobs:
        bufs[mid].zero_()
        rt.rt_trace(ctx, grids[mid], src, opt, bufs[mid], **prm)
    torch.cuda.synchronize()
    serial = time.perf_counter() - t1
    for g in grids:
        g.close()
    del bufs
    # capacity: the same jobs submitted at once (served back to back, batched)
    srv = server()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    ts = [srv.submit(mid, src, opt, **prm) for (t_arr, mid, src, opt, prm) in jobs]
    for t in ts:
        srv.wait(t, 3600)
        srv.release(t)
    burst = time.perf_counter() - t2
    srv.close()
    return {"jobs": n_jobs, "seconds": float(arrivals[-1]), "rate_per_s": rate,
            "packets_per_job": f"log-uniform 1e5..{max_packets:.0e}", "wavelengths_per_job": "uniform 1..30",
            "slots": slots, "max_batch_jobs": max_batch_jobs, "max_batch_packets": int(max_batch_packets),
            "batch_window_ms": batch_window_ms, "packets_total": int(pk),
            "offered_packets_per_s": pk / float(arrivals[-1]),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "served_packets_per_s": pk / wall, "served_wall_s": wall,
            "burst_packets_per_s": pk / burst, "burst_wall_s": burst,
            "serial_packets_per_s": pk / serial, "serial_busy_s": serial,
            "burst_over_serial": serial / burst, "library": [m.name for m in library]}


def run_serve(a, rt, synth, ctx, torch):
    t0 = time.perf_counter()
    clk = _clock_start()
    res = serve_measure(rt, synth, ctx, torch, a.serve_seconds, a.serve_rate, a.serve_max_packets,
                        slots=a.serve_slots, max_batch_jobs=a.serve_batch, max_batch_packets=a.serve_batch_packets)
    clocks = clk.stop()
    line = {"metric": "serving: p50/p99 job latency and packages/s under Poisson arrivals",
            "workload": "serve", **res, "clocks": clocks, "wall_s": time.perf_counter() - t0}
    print(json.dumps(line))


def _peel_compare(rt, ctx, torch, m, obs, kw, configs, reps):
    """Exact peel-off once, then the tabulated one for each (block, tiles)."""
    g = rt.Grid(ctx, m.tree)
    nl = m.optics.n_lambda
    ab = torch.zeros((nl, g.n_cells), dtype=torch.float64, device="cuda")
    im_e = torch.zeros((obs.n_obs, nl, obs.ny, obs.nx), dtype=torch.float64, device="cuda")
    im_t = torch.zeros_like(im_e)
    le = None
    for _ in range(reps):
        im_e.zero_()
        le = rt.rt_peel(ctx, g, m.sources, m.optics, obs, im_e, ab, **kw)
    e = im_e.sum(dim=1).cpu().numpy()  # per observer, all bins
    mask = e > 1e-3 * e.max()
    out = {"cells": int(m.tree.n_cells), "observers": obs.n_obs, "scatterings": le["n_scatter"],
           "exact": {"peel_ms": le["peel_ms"], "peel_crossings": le["n_peel_cross"], "trace_ms": le["kernel_ms"]},
           "tabulated": []}
    for block, tiles in configs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tab = rt.PeelTables(ctx, g, obs, block, tiles)
        torch.cuda.synchronize()
        t_tab = (time.perf_counter() - t0) * 1e3
        lt = None
        for _ in range(reps):
            im_t.zero_()
            lt = rt.rt_peel_tabulated(ctx, g, m.sources, m.optics, obs, tab, im_t, ab, **kw)
        t = im_t.sum(dim=1).cpu().numpy()
        rel = (t[mask] - e[mask]) / e[mask]
        out["tabulated"].append({
            "block_edge": block, "tiles_per_edge": tiles, "table_entries": tab.size, "table_build_ms": t_tab,
            "deferred": lt["n_peel_deferred"], "peel_ms": lt["peel_ms"], "peel_crossings": lt["n_peel_cross"],
            "peel_speedup": le["peel_ms"] / lt["peel_ms"] if lt["peel_ms"] else None,
            "total_speedup": (le["peel_ms"] + le["kernel_ms"]) / (lt["peel_ms"] + lt["kernel_ms"]),
            "image_rel_rms_bright_pixels": float(np.sqrt(np.mean(rel ** 2))),
            "image_rel_median_abs_bright_pixels": float(np.median(np.abs(rel))),
            "flux_ratio": float(t.sum() / e.sum())})
        tab.close()
    return out


def run_peeltab(a, rt, synth, ctx, torch):
    kw = dict(seed=1006, precision=32, rr_wmin=1e-4, rr_p=0.9)
    cloud = synth.cloud(n_root=a.n_root, levels=a.levels, n_lambda=a.n_lambda, packets_per_bin=0, n_pix=a.n_pix)
    res_c = _peel_compare(rt, ctx, torch, cloud, cloud.observers, dict(kw, packets_per_bin=2_000_000),
                          [(8, 8), (8, 32), (16, 64)], max(1, a.steps))
    disc = synth.disc(packets=0)
    box = disc.tree.box[0]
    el = np.deg2rad(2.0)
    az = np.deg2rad(np.arange(5) * 72.0)
    dirs = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.full(5, np.sin(el))], axis=1)
    obs = synth.Observers(dirs=dirs, ups=np.tile([0.0, 0.0, 1.0], (5, 1)), nx=256, ny=256, fov=(box, box))
    res_d = _peel_compare(rt, ctx, torch, disc, obs, dict(kw, packets_total=20_000_000),
                          [(8, 8), (8, 64), (4, 64), (2, 32)], max(1, a.steps))
    print(json.dumps({"metric": "accelerated peel-off (extinction tables) vs exact peel-off marches",
                      "workload": "peeltab", "cloud": res_c, "disc": res_d, "dtype": "f32"}))


def run_split(a, rt, synth, ctx, torch):
    """Table 1: noise of the 4 um field per hierarchy level with and without
    resampling, R runs each from the same initial packages (seeds differ),
    deviations taken from the mean of all 2R runs of a source type."""
    cloud = synth.cloud(n_root=a.n_root, levels=a.levels, n_lambda=1, packets_per_bin=0, n_pix=16)
    desc = cloud.tree
    L = desc.box[0]
    rho_unit = 70.0 * 2.8 * synth.MH_G
    kV = 0.4 / (rho_unit * L)
    lam = np.array([a.split_lambda])
    optics = synth.Optics(lambda_um=lam, kappa_ext=kV * (lam / 0.55) ** -1.8, albedo=synth.albedo_law(lam),
                          g_hg=np.array([0.5]), dnu=np.ones(1))
    # embedded sources: point sources at the centres of the four densest root cells
    n0 = int(np.prod(desc.root))
    h = L / desc.root[0]
    top = np.argsort(desc.density[:n0])[-4:]
    stars = [synth.Source("point", bin_energy=np.array([0.25]),
                          pos=((i % desc.root[0] + 0.5) * h, ((i // desc.root[0]) % desc.root[1] + 0.5) * h,
                               (i // (desc.root[0] * desc.root[1]) + 0.5) * h)) for i in top]
    ext = [synth.Source("external", bin_energy=np.array([1.0]))]
    g = rt.Grid(ctx, desc)
    lev = synth_levels(desc)
    leaf = desc.refine_flags == 0
    vol = (h * 0.5 ** lev) ** 3
    mass = torch.as_tensor(desc.density * vol, device="cuda:0")
    runs = max(2, a.split_runs)
    npk = a.split_packets
    clk = _clock_start()
    out = {}
    for name, src in (("external", ext), ("internal", stars)):
        res = {}
        J = {}
        for N in (1, 4):
            s1 = torch.zeros(g.n_cells, dtype=torch.float64, device="cuda:0")
            s2 = torch.zeros_like(s1)
            ab = torch.zeros((1, g.n_cells), dtype=torch.float64, device="cuda:0")
            ms, nsplit, ncross = [], 0, 0
            for r in range(runs + 1):
                ab.zero_()
                led = rt.rt_trace(ctx, g, src, optics, ab, seed=3000 + r, precision=32, packets_per_bin=npk,
                                  rr_wmin=1e-4, rr_p=0.9, split_factor=N)
                if r == 0:
                    continue  # warm-up
                ms.append(led["kernel_ms"])
                nsplit += led["n_split"]
                ncross += led["n_cross"]
                assert led["n_split_skipped"] == 0
                j = ab[0] / mass
                s1 += j
                s2 += j * j
            res[N] = dict(trace_ms=float(np.median(ms)), n_split=nsplit // runs, n_cross=ncross // runs)
            J[N] = (s1, s2)
        ref = (J[1][0] + J[4][0]) / (2 * runs)
        noise = {}
        for N in (1, 4):
            s1, s2 = J[N]
            # mean over runs of (J - J_ref)^2 per cell
            msd = (s2 - 2 * ref * s1 + runs * ref * ref) / runs
            msd = msd.cpu().numpy()
            noise[N] = [float(np.sqrt(np.mean(msd[leaf & (lev == l)]))) if np.any(leaf & (lev == l)) else None
                        for l in range(int(lev.max()) + 1)]
        top_n = max(v for N in (1, 4) for v in noise[N] if v is not None)
        worst1 = max(v for v in noise[1] if v is not None)
        worst4 = max(v for v in noise[4] if v is not None)
        out[name] = {"levels": list(range(int(lev.max()) + 1)),
                     "rms_with_resampling": [None if v is None else round(v / top_n, 4) for v in noise[4]],
                     "rms_no_resampling": [None if v is None else round(v / top_n, 4) for v in noise[1]],
                     "trace_ms_with": res[4]["trace_ms"], "trace_ms_without": res[1]["trace_ms"],
                     "copies_per_run": res[4]["n_split"],
                     "crossings_per_run_with": res[4]["n_cross"], "crossings_per_run_without": res[1]["n_cross"],
                     # packages needed without resampling for the worst level's noise with it, in time
                     "equal_noise_speedup": float((worst1 / worst4) ** 2 * res[1]["trace_ms"] / res[4]["trace_ms"])}
    clocks = clk.stop()
    print(json.dumps({"metric": f"resampling at grid boundaries (Table 1): RMS noise per level, {a.split_lambda:g} um field",
                      "workload": "split", "cells": int(g.n_cells), "runs": runs, "packages_per_run": npk,
                      "split_factor": 4, **out, "dtype": "f32", "clocks": clocks}))


def run_merge(a, rt, synth, ctx, torch):
    """Sect. 4.1: full resolution against the hierarchical model built from
    it, traced with the same packages (same seed), scattered-light maps
    compared by Eqs. 6-7."""
    n_full, root_n = 256, 32
    box_pc = 2.0
    L = box_pc * synth.PC_CM
    rho_unit = 70.0 * 2.8 * synth.MH_G
    g = synth.gaussian_random_field(n_full, 1002)
    rho = rho_unit * np.exp(1.5 * g - 1.125)          # [z][y][x], mean rho_unit
    lam = np.array([0.3, 0.55, 1.0, 2.2])[: max(1, min(4, a.n_lambda))]  # scattered light: UV to near-IR
    kV = 0.4 / (rho_unit * L)                          # mean tau_V across the box = 0.4
    optics = synth.powerlaw_dust(lam, kV, 0.55, g=0.5)
    src = [synth.Source("external", bin_energy=np.full(lam.size, 1.0 / lam.size))]
    obs = synth.axis_observers(n_full, L, "all6")
    full = synth.TreeDesc(root=(n_full,) * 3, box=(L,) * 3, n_refined=np.zeros(1, np.int64),
                          refine_flags=np.zeros(n_full ** 3, np.uint8), density=rho.ravel().copy())
    rho_dev = torch.from_numpy(rho).to("cuda:0")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    amr = rt.rt_merge_uniform(ctx, rho_dev, (root_n,) * 3, (L,) * 3, kV, 0.05, 30.0)
    merge_s = time.perf_counter() - t0
    del rho_dev
    npk = a.merge_packets
    clk = _clock_start()
    res = {}
    # the full model twice (other seed: the Monte Carlo noise floor of the
    # comparison), then the hierarchical model with the first seed
    for name, desc, seed in (("full", full, 1001), ("full_seed2", full, 2002), ("hierarchical", amr, 1001)):
        gr = rt.Grid(ctx, desc)
        im = torch.zeros((obs.n_obs, lam.size, obs.ny, obs.nx), dtype=torch.float64, device="cuda:0")
        ms = []
        for r in range(max(1, a.steps) + 1):
            im.zero_()
            led = rt.rt_peel(ctx, gr, src, optics, obs, im, None, seed=seed, precision=32, packets_per_bin=npk,
                             rr_wmin=1e-4, rr_p=0.9)
            if r:
                ms.append(led["kernel_ms"] + led["peel_ms"])
        res[name] = dict(cells=int(gr.n_cells), ms=float(np.median(ms)), n_cross=int(led["n_cross"]),
                         n_peel_cross=int(led["n_peel_cross"]), images=im.cpu().numpy())
        del gr
    clocks = clk.stop()
    f, h, f2 = res["full"]["images"], res["hierarchical"]["images"], res["full_seed2"]["images"]
    per_lambda = []
    def binned(x, k=8):  # k x k pixel blocks: less Monte Carlo noise per map element
        o, ny, nx = x.shape
        return x.reshape(o, ny // k, k, nx // k, k).sum(axis=(2, 4))

    for b in range(lam.size):
        d = h[:, b] - f[:, b]
        n = f2[:, b] - f[:, b]
        fb, db, nb = binned(f[:, b]), binned(d), binned(n)
        per_lambda.append({"lambda_um": float(lam[b]),
                           "delta_mean": float(d.sum() / f[:, b].sum()),
                           "delta_rms": float(np.sqrt((d * d).sum() / (f[:, b] ** 2).sum())),
                           "noise_floor_delta_mean": float(n.sum() / f[:, b].sum()),
                           "noise_floor_delta_rms": float(np.sqrt((n * n).sum() / (f[:, b] ** 2).sum())),
                           "delta_rms_8x8": float(np.sqrt((db * db).sum() / (fb * fb).sum())),
                           "noise_floor_delta_rms_8x8": float(np.sqrt((nb * nb).sum() / (fb * fb).sum()))})
    print(json.dumps({"metric": "hierarchical model built from the full-resolution cube (Sect. 4.1)",
                      "workload": "merge", "full_cells": res["full"]["cells"],
                      "hierarchical_cells": res["hierarchical"]["cells"],
                      "cell_ratio": res["full"]["cells"] / res["hierarchical"]["cells"],
                      "levels": int(amr.n_levels), "cells_per_level_refined": [int(v) for v in amr.n_refined],
                      "merge_s": merge_s, "packages_per_bin": npk, "n_lambda": int(lam.size),
                      "trace_peel_ms_full": res["full"]["ms"], "trace_peel_ms_hierarchical": res["hierarchical"]["ms"],
                      "speedup": res["full"]["ms"] / res["hierarchical"]["ms"],
                      "crossings_full": res["full"]["n_cross"], "crossings_hierarchical": res["hierarchical"]["n_cross"],
                      "peel_crossings_full": res["full"]["n_peel_cross"],
                      "peel_crossings_hierarchical": res["hierarchical"]["n_peel_cross"],
                      "maps": per_lambda, "dtype": "f32", "clocks": clocks}))


def run_poly(a, rt, synth, ctx, torch):
    """Polychromatic against monochromatic packages at the same number of
    packages per wavelength bin (monochromatic) or per group (polychromatic),
    untiled, FP32.  Noise: relative RMS difference of two seeds per bin."""
    m = synth.cloud(n_root=128, levels=3, n_lambda=20, packets_per_bin=0, n_pix=64)
    ctx.set_tiles(0)
    g = rt.Grid(ctx, m.tree)
    nl = m.optics.n_lambda
    obs = m.observers
    leaf = torch.as_tensor(m.tree.refine_flags == 0, device="cuda:0")
    npk = a.poly_packets
    clk = _clock_start()
    out = {}
    # the summed absorbed energy (what the temperature solve takes): one
    # accumulator update per crossing and group instead of one per bin
    summed = {}
    for F in (1, a.poly_group):
        ab = torch.zeros((1, g.n_cells), dtype=torch.float64, device="cuda:0")
        t = []
        for seed in (11, 22):
            ab.zero_()
            led = rt.rt_trace(ctx, g, m.sources, m.optics, ab, seed=seed, precision=32, packets_per_bin=npk,
                              rr_wmin=1e-4, rr_p=0.9, poly_group=F, per_lambda=False)
            t.append(led["kernel_ms"])
        summed[F] = float(t[-1])
    for F in (1, a.poly_group):
        runs = []
        for seed in (11, 22, 33):
            ab = torch.zeros((nl, g.n_cells), dtype=torch.float64, device="cuda:0")
            im = torch.zeros((obs.n_obs, nl, obs.ny, obs.nx), dtype=torch.float64, device="cuda:0")
            led = rt.rt_peel(ctx, g, m.sources, m.optics, obs, im, ab, seed=seed, precision=32, packets_per_bin=npk,
                             rr_wmin=1e-4, rr_p=0.9, poly_group=F)
            runs.append((ab[:, leaf], im, led))
        ms = float(np.median([r[2]["kernel_ms"] + r[2]["peel_ms"] for r in runs[1:]]))
        a1, a2 = runs[1][0], runs[2][0]
        i1, i2 = runs[1][1], runs[2][1]
        cell_noise = (torch.sqrt(((a1 - a2) ** 2).mean(dim=1) / 2) / a1.abs().mean(dim=1).clamp_min(1e-300)).cpu().numpy()
        img_noise = (torch.sqrt(((i1 - i2) ** 2).sum(dim=(0, 2, 3)) / 2 / (i1 ** 2).sum(dim=(0, 2, 3)).clamp_min(1e-300))
                     ).cpu().numpy()
        out[F] = dict(ms=ms, packages=int(runs[1][2]["n_packets"]), crossings=int(runs[1][2]["n_cross"]),
                      peel_crossings=int(runs[1][2]["n_peel_cross"]), cell_noise=cell_noise, img_noise=img_noise,
                      absorbed_total=runs[1][0].sum(dim=1).cpu().numpy())
    clocks = clk.stop()
    P = a.poly_group
    eff_cells = (out[1]["ms"] * out[1]["cell_noise"] ** 2) / (out[P]["ms"] * out[P]["cell_noise"] ** 2)
    eff_img = (out[1]["ms"] * out[1]["img_noise"] ** 2) / (out[P]["ms"] * np.maximum(out[P]["img_noise"], 1e-300) ** 2)
    print(json.dumps({
        "metric": "polychromatic packages (Sect. 2.3) against monochromatic ones",
        "workload": "poly", "cells": int(g.n_cells), "n_lambda": nl, "group": P,
        "packages_per_bin_or_group": npk,
        "ms_mono": out[1]["ms"], "ms_poly": out[P]["ms"],
        "trace_ms_summed_output_mono": summed[1], "trace_ms_summed_output_poly": summed[P],
        "packages_mono": out[1]["packages"], "packages_poly": out[P]["packages"],
        "crossings_mono": out[1]["crossings"], "crossings_poly": out[P]["crossings"],
        "peel_crossings_mono": out[1]["peel_crossings"], "peel_crossings_poly": out[P]["peel_crossings"],
        "lambda_um": [float(v) for v in m.optics.lambda_um],
        "cell_noise_mono": [round(float(v), 5) for v in out[1]["cell_noise"]],
        "cell_noise_poly": [round(float(v), 5) for v in out[P]["cell_noise"]],
        "image_noise_mono": [round(float(v), 5) for v in out[1]["img_noise"]],
        "image_noise_poly": [round(float(v), 5) for v in out[P]["img_noise"]],
        "absorbed_ratio_poly_over_mono": [round(float(x / y), 5) if y > 0 else None
                                          for x, y in zip(out[P]["absorbed_total"], out[1]["absorbed_total"])],
        "efficiency_cells": [round(float(v), 3) for v in eff_cells],
        "efficiency_images": [round(float(v), 3) for v in eff_img],
        "dtype": "f32", "clocks": clocks}))
