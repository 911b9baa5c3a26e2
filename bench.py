#!/usr/bin/env python
"""Throughput of the batched scintillation pipeline on GB300: one JSON line on rank 0.

Workload (default "batched"): 48 seeded screens, 16 each of 1024^2, 2048^2 and
4096^2 (10 km pixels, R_diff ~ U[30, 300] km at 550 nm, Kolmogorov), each
propagated at 32 wavelengths in 400-700 nm (flat passband), smoothed by a
projected stellar disk of U[0.1, 2] R_ref and sampled along 8 straight tracks,
with the modulation index of the map and of every curve.  A step is one pass of
the whole hot path over the batch: synthesis -> passband propagation ->
smoothing -> light curves -> modulation indices, issued by scint_run_batch on
eight internal streams and replayed as one CUDA graph.

Metric: Fresnel-propagated pixels per second, sum over screens of N^2 x
N_lambda per step / step time.  Timing: CUDA events on the launching stream,
barrier + synchronize around exactly --steps replays after --warmup untimed
ones, max over ranks.  Every per-screen field is 32-134 MB and a step moves
hundreds of GB, so the inputs exceed the 129 MB L2 between steps.

Multi-GPU: independent batches per rank (seeds offset by rank), no collective
on the data path: weak scaling.  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Fresnel-propagated pixels/sec, batched FP32 vs plain, at <=2e-4 err; %HBM peak"
UNIT = "pixel-wavelengths/s"
PARAM_KEYS = ("n", "pixel_km", "r_diff_km", "beta", "lambda_nm", "lambda_ref_nm", "z_pc",
              "source_radius_km", "seed", "screen_id", "margin_km")
CPU_SAMPLE_N = 2048       # the batch screen the oracle is timed on (about 10 s on one core)
FP32_LANES_PER_SM = 128


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def _sm_count() -> int:
    """SMs of the current CUDA device (from its properties)."""
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def _workload(name: str, rank: int, screens: int = 1):
    from paper_1301_0514_gb300 import workloads as W
    if name == "batched":
        items = W.batched_polychromatic()
        desc = ("batched: 48 screens (16 each of 1024^2, 2048^2, 4096^2, 10 km pixels, R_diff U[30,300] km) "
                "x 32 wavelengths 400-700 nm, disk sources U[0.1,2] R_ref, 8 tracks/screen")
    elif name == "profile":
        items = [x for x in W.batched_polychromatic() if x["n"] == 4096][:screens]
        for it in items:
            it["lambdas_nm"] = it["lambdas_nm"][::4]
        desc = (f"profiling case: {len(items)} 4096^2 screen(s) of the batched workload x 8 wavelengths "
                f"(~{1.2 * len(items):.1f} GB on the device, above the L2 size)")
    elif name == "large16384":
        items = [W.large_screen_16384(beta=11.0 / 3.0, disk=True)]
        desc = ("one 16384^2 screen (lines split over two-block clusters), 5 km pixels, R_diff 100 km, "
                "Kolmogorov, 500 nm, disk of one R_ref")
    else:
        items = W.single_screens_4096(r_diffs=(100.0,))
        items[0]["lambdas_nm"] = np.array([500.0])
        desc = "single 4096^2 screen, 10 km pixels, R_diff 100 km, 500 nm, point source, 64 tracks"
    for it in items:
        it["seed"] += 100000 * rank
    return items, desc


def _max_over_ranks(ms: float, world: int, device) -> float:
    """The step time of the job: the slowest rank's (all-reduce MAX; identity on one rank)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _kernel_source_hash(files):
    """Hash of the CUDA sources a kernel is built from (a traffic record is void once they change)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1301_0514_gb300", "csrc")
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"scint_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _cufft_comparison(items, dev, lams_every=4):
    """The same passband propagation of one 4096^2 screen from library FFTs: torch's cuFFT
    fft2/ifft2 plus elementwise tensor ops (phase reduced mod 2 pi in FP64, field and FFTs in
    complex64), timed with CUDA events, and its map compared with this library's.  A
    comparison only: it is not the product path."""
    import torch
    import paper_1301_0514_gb300 as S
    it = [x for x in items if x["n"] == 4096][0]
    p = S.params(**{k: it[k] for k in PARAM_KEYS})
    lams = it["lambdas_nm"][::lams_every]
    w = np.full(len(lams), 1.0 / len(lams))
    n = p.n
    L = n * p.pixel_km
    phi = S.make_screen(p)
    ours = S.sum_passband(p, phi, lams, w)
    k = torch.fft.fftfreq(n, d=p.pixel_km, dtype=torch.float64, device=dev)
    x = (torch.arange(n, dtype=torch.float64, device=dev) + 0.5) * p.pixel_km
    stream = torch.cuda.current_stream(dev)

    def tables(lam):
        lz = lam * 1e-12 * p.z_pc * 3.0856775814913673e13
        lm = min(10.0 * np.sqrt(lz / (2 * np.pi)), L / 4) if p.margin_km < 0 else p.margin_km
        u = torch.minimum(x, L - x)
        sf = torch.where(u <= lm, torch.sin(np.pi * u / (2 * lm)) ** 2, torch.ones_like(u)) if lm > 0 else torch.ones_like(u)
        turns = lz * k * k / 2.0
        ph = -2.0 * np.pi * (turns - torch.round(turns))
        h = torch.polar(torch.ones_like(ph), ph).to(torch.complex64)
        return sf.float(), h

    tab = [tables(l) for l in lams]

    def run():
        out = torch.zeros((n, n), dtype=torch.float32, device=dev)
        for (sf, h), lam, wl in zip(tab, lams, w):
            turns = phi * (p.lambda_ref_nm / lam) / (2 * np.pi)
            a = torch.polar(torch.ones((n, n), dtype=torch.float32, device=dev),
                            (2 * np.pi * (turns - torch.round(turns))).float())
            a = a * (sf[:, None] * sf[None, :])
            f = torch.fft.ifft2(torch.fft.fft2(a) * (h[:, None] * h[None, :]))
            out += float(wl) * (f.real ** 2 + f.imag ** 2)
        return out

    run()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = run()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    e0.record(stream)
    S.sum_passband(p, phi, lams, w, out=ours)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_ours = e0.elapsed_time(e1)
    units = float(n) * n * len(lams)
    return {"value": units / (ms * 1e-3), "ms": ms, "unit": UNIT, "ours_value": units / (ms_ours * 1e-3),
            "ours_ms": ms_ours, "max_abs_diff": float((res - ours).abs().max().item()),
            "form": f"one 4096^2 screen x {len(lams)} wavelengths: torch cuFFT fft2/ifft2 + elementwise ops, "
                    f"against scint_sum_passband on the same screen"}


def _oracle_ready(_):
    """Pool warm-up: the worker imports the oracle before the timed region."""
    import oracle  # noqa: F401
    return os.getpid()


def _oracle_partial(task):
    """One worker's share of the all-core oracle run: the weighted passband sum over a
    subset of the wavelengths (weights are absolute, so the partial sums add up)."""
    import oracle as O
    phi, pkw, lams, w = task
    return O.sum_passband(phi, O.ScreenParams(**pkw), lams, w)


def _cpu_baseline(items, gpu_maps):
    """FP64 oracle on one 2048^2 screen of the batch (all 32 wavelengths, disk, tracks): on all
    host cores (the wavelengths spread over spawned worker processes, the screen, smoothing and
    curves in the parent) and on one core."""
    import oracle as O
    it = [x for x in items if x["n"] == CPU_SAMPLE_N][0]
    pkw = {k: it[k] for k in PARAM_KEYS}
    p = O.ScreenParams(**pkw)
    lams = np.asarray(it["lambdas_nm"], dtype=np.float64)
    w = (np.full(lams.size, 1.0 / lams.size) if it["weights"] is None
         else np.asarray(it["weights"], dtype=np.float64))
    units = p.n * p.n * lams.size

    def finish(I):
        I = O.smooth_source(I, p.pixel_km, p.source_radius_km)
        curves = O.lightcurves(I, it["tracks"], it["n_samples"])
        m_map = O.modulation_index_map(I, p)
        [O.modulation_index(c) for c in curves]
        return I, m_map

    t0 = time.perf_counter()
    phi = O.make_screen(p)
    I, m_map = finish(O.sum_passband(phi, p, lams, w))
    dt = time.perf_counter() - t0
    single = {"value": units / dt, "cores": 1,
              "sample": f"one {p.n}^2 screen of the batch x {lams.size} wavelengths + disk + "
                        f"{len(it['tracks'])} tracks, {dt:.1f} s"}
    out = {"value": single["value"], "unit": UNIT, "cores": 1, "kind": "oracle", "sample": single["sample"]}
    workers = min(os.cpu_count() or 1, lams.size)
    if workers > 1:
        import multiprocessing as mp
        chunks = np.array_split(np.arange(lams.size), workers)
        # spawn: this process has a CUDA context, and a forked child of it can hang
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_oracle_ready, range(workers))
            t0 = time.perf_counter()
            phi_p = O.make_screen(p)
            parts = pool.map(_oracle_partial, [(phi_p, pkw, lams[c], w[c]) for c in chunks])
            I_p, m_p = finish(np.sum(parts, axis=0))
            dt_p = time.perf_counter() - t0
        out = {"value": units / dt_p, "unit": UNIT, "cores": workers, "kind": "oracle",
               "sample": f"the same screen with its {lams.size} wavelengths spread over {workers} worker "
                         f"processes ({dt_p:.1f} s; screen, smoothing and curves in the parent)",
               "single_core": single,
               "all_core_vs_single_max_abs_diff": float(np.abs(I_p - I).max())}
    err = None
    if gpu_maps is not None and it["seed"] in gpu_maps:
        g_I, g_m = gpu_maps[it["seed"]]
        err = {"max_abs_intensity_err": float(np.abs(g_I - I).max()),
               "m_rel_err": float(abs(g_m - m_map) / m_map)}
    return out, err


def run_reference(args):
    rank, world, local = _dist()
    if rank != 0:
        return
    items, desc = _workload(args.workload, 0)
    import oracle as O
    it = [x for x in items if x["n"] == min(x["n"] for x in items)][0]
    p = O.ScreenParams(**{k: it[k] for k in PARAM_KEYS})
    lams = it["lambdas_nm"][:4]        # bounded sample per step: 4 wavelengths of one screen

    def step():
        phi = O.make_screen(p)
        I = O.sum_passband(phi, p, lams)
        if p.source_radius_km > 0:
            I = O.smooth_source(I, p.pixel_km, p.source_radius_km)
        O.lightcurves(I, it["tracks"], it["n_samples"])
        return I

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = p.n * p.n * len(lams) / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "sample": f"one {p.n}^2 screen x {len(lams)} wavelengths per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"one {p.n}^2 screen x {len(lams)} wavelengths per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_1301_0514_gb300 as S

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    items, desc = _workload(args.workload, rank, args.profile_screens)
    P = [S.params(**{k: it[k] for k in PARAM_KEYS}) for it in items]
    sizes = sorted({p.n for p in P})
    lams, wts = items[0]["lambdas_nm"], items[0]["weights"]
    assert all(np.array_equal(it["lambdas_nm"], lams) for it in items), "one passband per batch"
    n_lam = len(lams)
    curves = [torch.empty((len(it["tracks"]), it["n_samples"]), dtype=torch.float32, device=dev) for it in items]
    m_map = torch.empty((len(items), 4), dtype=torch.float64, device=dev)
    m_curve = [torch.empty((len(it["tracks"]), 3), dtype=torch.float64, device=dev) for it in items]
    # the screen checked against the oracle keeps its intensity map; the others live in lane scratch
    par_i = next((i for i, p in enumerate(P) if p.n == CPU_SAMPLE_N), None)
    par_I = (torch.empty((CPU_SAMPLE_N, CPU_SAMPLE_N), dtype=torch.float32, device=dev)
             if par_i is not None else None)
    entries = [dict(params=p, tracks=it["tracks"], n_samples=it["n_samples"], curves=curves[i],
                    m_map=m_map[i], m_curves=m_curve[i], intensity=par_I if i == par_i else None)
               for i, (p, it) in enumerate(zip(P, items))]
    batch = S.batch_items(entries)
    old_mode = S.batch_mode(1)        # the persistent form needs the larger workspace
    ws_persist = S.batch_workspace_bytes(batch, n_lam, args.lanes)
    S.batch_mode(old_mode)
    ws = torch.empty(max(S.batch_workspace_bytes(batch, n_lam, args.lanes), ws_persist,
                         max(S.workspace_bytes(p, 1) for p in P)), dtype=torch.uint8, device=dev)
    # plain form: its own maps, one per grid size
    phi = {n: torch.empty((n, n), dtype=torch.float64, device=dev) for n in sizes}
    inten = {n: torch.empty((n, n), dtype=torch.float32, device=dev) for n in sizes}
    units = sum(p.n * p.n * len(it["lambdas_nm"]) for p, it in zip(P, items))
    stream = torch.cuda.current_stream(dev)

    def plain_screen(i, p, it):
        S.make_screen(p, out=phi[p.n], workspace=ws)
        w = wts if wts is not None else np.full(n_lam, 1.0 / n_lam)
        for j, lam in enumerate(lams):
            S.sum_passband(p, phi[p.n], [lam], [w[j]], out=inten[p.n], accumulate=j > 0, workspace=ws)
        S.smooth_source(p, inten[p.n], workspace=ws)
        S.lightcurve(p, inten[p.n], it["tracks"], it["n_samples"], out=curves[i])
        S.modulation_index(p, inten[p.n], out=m_map[i], workspace=ws)
        S.curve_modulation(curves[i], out=m_curve[i])

    def step(plain=False):
        if plain:
            for i, (p, it) in enumerate(zip(P, items)):
                plain_screen(i, p, it)
        else:
            S.run_batch(batch, lams, wts, n_lanes=lanes, workspace=ws)

    # propagation plans: the autotuner times the built variants per grid size (outside capture),
    # or a fixed choice (--plans unpacked / packed)
    lanes = args.lanes
    tuned_batch = None
    if args.batch_mode != "tune":
        S.batch_mode(1 if args.batch_mode == "persistent" else 0)
    if args.plans == "tune":
        # the batch tuner times the whole batch under candidate plan sets and lane counts
        lanes, tuned_ms, mode = S.tune_batch(batch, lams, wts, workspace=ws)
        tuned_batch = {"lanes": lanes, "ms": tuned_ms, "mode": "persistent" if mode == 1 else "lanes"}
        plans = {str(n): S.get_plan(n) for n in sizes}
    else:
        for n in sizes:
            S.set_plan(n, 1 if args.plans == "packed" else 0, 2, 2 if args.plans == "packed" else 1, 16)
        plans = {str(n): S.get_plan(n) for n in sizes}
    # warm-up outside the graph (sets kernel attributes), then capture one graph of the step
    step()
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="relaxed"):
        step()
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = _max_over_ranks(ms, world, dev)
    value = units * world / (ms * 1e-3)

    # Per-kernel times: concurrent lanes share the SMs, so an event pair around a
    # launch would also count other lanes' kernels.  The kernels are timed in a
    # serial replay of the same step (one lane, event pairs as graph nodes).
    S.profile_enable(True)
    pgraph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(pgraph, capture_error_mode="relaxed"):
        S.run_batch(batch, lams, wts, n_lanes=1, workspace=ws)
    torch.cuda.synchronize(dev)
    pgraph.replay()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    pgraph.replay()
    q1.record(stream)
    torch.cuda.synchronize(dev)
    ms_serial = q0.elapsed_time(q1)
    kstats = S.profile_read()           # per-kernel event times of the last serial replay
    S.profile_enable(False)

    # plain form: one screen and one wavelength per call, no graph, same kernels; one untimed
    # pass, then --steps timed passes
    step(plain=True)
    torch.cuda.synchronize(dev)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        step(plain=True)
    p1.record(stream)
    torch.cuda.synchronize(dev)
    ms_plain = p0.elapsed_time(p1) / args.steps

    cufft = _cufft_comparison(items, dev) if any(it["n"] == 4096 for it in items) else None

    # end to end through the public API with host inputs and host results
    pinned_curves = [torch.empty(c.shape, dtype=c.dtype, pin_memory=True) for c in curves]
    pinned_m = torch.empty(m_map.shape, dtype=m_map.dtype, pin_memory=True)
    h2d = sum(it["tracks"].nbytes + it["lambdas_nm"].nbytes + 96 for it in items)
    d2h = sum(c.numel() * 4 for c in curves) + m_map.numel() * 8
    e2e_steps = args.steps
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step()
        for c, pc in zip(curves, pinned_curves):
            pc.copy_(c, non_blocking=True)
        pinned_m.copy_(m_map, non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps

    # roofline of the dominant kernel (largest share of the timed step)
    hbm_peak, sm_max_mhz, peak_src = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak_tflops = sm_count * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    dom_name, dom = max(kstats.items(), key=lambda kv: kv[1]["total_ms"])
    per_launch_ms = dom["total_ms"] / dom["launches"]   # from the serial replay
    gbs = dom["bytes"] / (dom["total_ms"] * 1e-3) / 1e9
    tflops = dom["flops"] / (dom["total_ms"] * 1e-3) / 1e12
    ridge = alu_peak_tflops * 1e12 / (hbm_peak * 1e9)
    intensity = dom["flops"] / dom["bytes"] if dom["bytes"] else 0.0
    traffic = None
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        rec = tr.get(dom_name)
        if rec and rec.get("source_hash") == _kernel_source_hash(rec["sources"]):
            # DRAM bytes of one captured launch scale with the lines it processes:
            # the captured dram/algorithmic ratio times this launch's algorithmic bytes
            traffic = rec["dram_over_algorithmic"] * dom["bytes"] / dom["launches"]
    except Exception:
        pass
    if intensity > ridge:
        roof = {"bound": "alu", "achieved": tflops, "peak": alu_peak_tflops, "unit": "TFLOP/s",
                "frac": tflops / alu_peak_tflops, "traffic": traffic}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "traffic": traffic}
    roof.update({"kernel": dom_name, "launch_ms": per_launch_ms, "share": dom["total_ms"] / ms_serial,
                 "timing": f"serial one-lane replay of the step ({ms_serial:.1f} ms), CUDA events per launch",
                 "algorithmic_bytes_per_launch": dom["bytes"] / dom["launches"],
                 "fft_flops_per_launch": dom["flops"] / dom["launches"], "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak,
                 "peak_source": f"hbm {peak_src} (MEASURED_PEAKS.json); alu = {sm_count} SMs (device) x "
                                f"{FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max_mhz:.0f} MHz"})
    # the same kernel and the whole step on the planning bytes: 24 B per pixel-wavelength per
    # propagation pass (48 for the pair), 24 B per pixel for the smoothing, 40 B per pixel for
    # the synthesis (a three-pass design's minimal traffic)
    px = sum(p.n * p.n for p in P)
    plan_step_bytes = 48.0 * units + 24.0 * sum(p.n * p.n for p in P if p.source_radius_km > 0) + 40.0 * px
    dom_px_lambda = units / max(1, dom["launches"]) if dom_name in ("prop_rows", "prop_cols") else None
    planning = {"step_bytes": plan_step_bytes, "step_GBps": plan_step_bytes / (ms * 1e-3) / 1e9,
                "step_frac": plan_step_bytes / (ms * 1e-3) / 1e9 / hbm_peak,
                "note": "planning bytes: 48 B per pixel-wavelength for propagation, 24 B/px smoothing, "
                        "40 B/px synthesis; the two-pass kernels move 16 B per pixel-wavelength"}
    if dom_px_lambda is not None:
        kb = 24.0 * dom_px_lambda / (per_launch_ms * 1e-3) / 1e9
        planning.update({"kernel_bytes_per_px_lambda": 24.0, "kernel_GBps": kb, "kernel_frac": kb / hbm_peak})
    roof["planning_bytes_hbm"] = planning
    launches = sum(v["launches"] for v in kstats.values())
    kernels = {k: {"launches": v["launches"], "ms": v["total_ms"], "share": v["total_ms"] / ms_serial,
                   "GBps": v["bytes"] / max(v["total_ms"], 1e-9) / 1e6,
                   "TFLOPs": v["flops"] / max(v["total_ms"], 1e-9) / 1e9} for k, v in kstats.items()}

    cpu = None
    err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and par_i is not None:
        it = items[par_i]
        step()
        torch.cuda.synchronize(dev)
        gmap = {it["seed"]: (par_I.cpu().numpy().astype(np.float64), float(m_map[par_i, 0].item()))}
        cpu, err = _cpu_baseline(items, gmap)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": desc, "form": f"scint_run_batch on {lanes} lane(s), one CUDA graph per step",
                           "plans": plans, "batch_tuner": tuned_batch,
                           "l2": "inputs larger than L2 (fields 32-134 MB per screen and wavelength)",
                           "parallelism": f"independent batch per GPU x{world}"},
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": units * world / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms},
                "gpu_launches": launches * args.steps, "clocks": clk,
                "serial": {"value": units / (ms_serial * 1e-3), "ms_per_step": ms_serial,
                           "form": "the same batch on one lane (kernels in sequence), with per-launch events"},
                "plain": {"value": units / (ms_plain * 1e-3), "ms_per_step": ms_plain, "steps": args.steps,
                          "form": "one screen at a time and one wavelength per call (no wavelength groups, no "
                                  "lanes, no graph) through the same fused kernels; the unfused form is "
                                  "cufft_comparison"},
                "three_pass_equivalent": {
                    "bytes_per_px_lambda": 48, "GBps": value / world * 48 / 1e9,
                    "frac_of_hbm": value / world * 48 / 1e9 / hbm_peak,
                    "note": "this throughput expressed in the bytes of a three-pass design (FFT_x | "
                            "FFT_y H IFFT_y | IFFT_x |A|^2, 48 B per pixel-wavelength); the two-pass "
                            "kernels move 16 B, so their own DRAM fraction is lower by design"},
                "cufft_comparison": cufft, "parity": err, "kernels": kernels}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_screen_check(args):
    """Sect. 3.1.1 screen check at the paper's size: S_rec over all annuli of one
    N x N realisation, D_rec at 256 lags and R_diff^rec.  Metric: spectral bins/s."""
    import torch
    import paper_1301_0514_gb300 as S
    from paper_1301_0514_gb300 import workloads as W

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    n, pix, rd = args.check_n, 28.85, 500.0
    p = S.params(n=n, pixel_km=pix, r_diff_km=rd, seed=W.SEED_BASE + 9100 + 100000 * rank)
    n_bins = S.max_annulus(n) + 1
    s = torch.empty(n_bins, dtype=torch.float64, device=dev)
    c = torch.empty(n_bins, dtype=torch.int64, device=dev)
    lags = torch.linspace(10.0, 0.25 * n * pix, 256, dtype=torch.float64, device=dev)
    d = torch.empty(256, dtype=torch.float64, device=dev)
    root = torch.empty(1, dtype=torch.float64, device=dev)
    ws = torch.empty(4096, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        S.spectrum_rec(p, out=(s, c))
        S.structure_function_rec(p, s, lags, workspace=ws, out=(d, root))

    step()
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="relaxed"):
        step()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = _max_over_ranks(ms, world, dev)
    units = float(n) * n
    value = units * world / (ms * 1e-3)

    # per-kernel times from one profiled eager step
    S.profile_enable(True)
    step()
    torch.cuda.synchronize(dev)
    kstats = S.profile_read()
    S.profile_enable(False)
    launches = sum(v["launches"] for v in kstats.values())
    dom_name, dom = max(kstats.items(), key=lambda kv: kv[1]["total_ms"])
    _, sm_max_mhz, _ = _peaks()
    # Philox4x32-10 bound: 10 rounds x 2 32x32->64-bit multiplies per bin, each a
    # multiply-add pair on the integer pipe (64 lanes per SM per clock)
    imad_per_bin = 40.0
    peak = _sm_count() * 64 * sm_max_mhz * 1e6 / imad_per_bin
    achieved = units / (kstats["radial_spectrum"]["total_ms"] * 1e-3)
    roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gbins/s",
            "frac": achieved / peak, "traffic": None, "kernel": "radial_spectrum",
            "peak_source": f"Philox4x32-10 integer multiplies: {_sm_count()} SMs x 64 lanes x {sm_max_mhz:.0f} MHz "
                           f"/ {imad_per_bin:.0f} per bin",
            "timing": "one profiled eager step, CUDA events per launch"}

    # end to end: the same calls with the results read back to pinned host memory
    hs = torch.empty(n_bins, dtype=torch.float64, pin_memory=True)
    hd = torch.empty(256 + 1, dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(3):
        step()
        hs.copy_(s, non_blocking=True)
        hd[:256].copy_(d, non_blocking=True)
        hd[256:].copy_(root, non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / 3

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        po = O.ScreenParams(n=n, pixel_km=pix, r_diff_km=rd, seed=p.seed)
        j_max = 1500          # about 4e7 of the 2e8 bins: several seconds of oracle time
        t0 = time.perf_counter()
        s_o, _ = O.spectrum_rec(po, j_max=j_max)
        dt = time.perf_counter() - t0
        rows = 2 * j_max + 1
        cpu = {"value": rows * n / dt, "unit": "bins/s", "cores": 1, "kind": "oracle",
               "sample": f"annulus sums over the {rows} spectral rows |m_y| <= {j_max} of the {n}^2 grid, {dt:.1f} s"}
        err = float(np.max(np.abs(s[:j_max + 1].cpu().numpy() - s_o) / np.maximum(np.abs(s_o), 1e-300)))
    if rank == 0:
        line = {"metric": f"screen-check spectral bins/s (Sect. 3.1.1, N={n})", "value": value, "unit": "bins/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
                "data": "synthetic",
                "config": {"workload": f"screen check: one {n}^2 realisation, 28.85 km pixels, R_diff 500 km, "
                                       f"{n_bins} annuli, D_rec at 256 lags, R_diff^rec by 64 bisection steps",
                           "l2": "no input: the noise is regenerated per bin"},
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": units * world / (e2e_ms * 1e-3), "unit": "bins/s", "h2d_bytes_per_step": 96,
                        "d2h_bytes_per_step": int(8 * (n_bins + 257)), "ms_per_step": e2e_ms},
                "gpu_launches": launches * args.steps, "clocks": clk,
                "r_diff_rec_km": float(root.item()),
                "parity": None if cpu is None else {"max_rel_err_low_annuli": err},
                "kernels": {k: {"launches": v["launches"], "ms": v["total_ms"]} for k, v in kstats.items()}}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_conjugate(args):
    """The paper's one-FFT propagator on a passband batch at critical sampling
    (N Delta^2 = lambda z at 550 nm), timed beside the transfer-function passband of
    the same screens.  Metric: pixel-wavelengths/s."""
    import torch
    import paper_1301_0514_gb300 as S
    from paper_1301_0514_gb300 import workloads as W

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    n, count = args.conj_n, 16
    lam_ref = 550.0
    pix = float(np.sqrt(lam_ref * W.KM_PER_NM * 160.0 * W.KM_PER_PC / n))
    lams = W.passband_400_700(32)
    rng = np.random.default_rng(W.SEED_BASE + 9400)
    P = [S.params(n=n, pixel_km=pix, r_diff_km=float(rng.uniform(3.0, 12.0) * pix), lambda_nm=lam_ref,
                  lambda_ref_nm=lam_ref, seed=W.SEED_BASE + 9400 + 100000 * rank + k, screen_id=k)
         for k in range(count)]
    phi = torch.empty((n, n), dtype=torch.float64, device=dev)
    out = torch.empty((n, n), dtype=torch.float32, device=dev)
    ws = torch.empty(S.workspace_bytes(P[0], len(lams)) + 4 * n * n * len(lams), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    units = float(n) * n * len(lams) * count

    def step(conj=True):
        for p in P:
            S.make_screen(p, out=phi, workspace=ws)
            if conj:
                S.sum_passband_conjugate(p, phi, lams, out=out, workspace=ws)
            else:
                S.sum_passband(p, phi, lams, out=out, workspace=ws)

    def timed(conj):
        step(conj)
        torch.cuda.synchronize(dev)
        S.profile_enable(True)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            step(conj)
        for _ in range(args.warmup):
            g.replay()
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ks = S.profile_read()
        S.profile_enable(False)
        return e0.elapsed_time(e1) / args.steps, ks

    clocks = ClockSampler(local)
    clocks.start()
    ms, kstats = timed(True)
    clk = clocks.stop()
    ms_tf, kstats_tf = timed(False)
    ms = _max_over_ranks(ms, world, dev)
    value = units * world / (ms * 1e-3)
    hbm_peak, sm_max_mhz, peak_src = _peaks()
    alu_peak = _sm_count() * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    dom_name, dom = max(((k, v) for k, v in kstats.items() if k.startswith("conj")), key=lambda kv: kv[1]["total_ms"])
    tflops = dom["flops"] / (dom["total_ms"] * 1e-3) / 1e12
    gbs = dom["bytes"] / (dom["total_ms"] * 1e-3) / 1e9
    roof = {"bound": "alu", "achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s", "frac": tflops / alu_peak,
            "traffic": None, "kernel": dom_name, "share": dom["total_ms"] / ms, "hbm_gbs": gbs,
            "hbm_frac": gbs / hbm_peak, "peak_source": f"alu = {_sm_count()} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                                       f"{sm_max_mhz:.0f} MHz; hbm {peak_src}"}

    # end to end through the public API: the passband map of every screen read back
    host = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for p in P:
        S.make_screen(p, out=phi, workspace=ws)
        S.sum_passband_conjugate(p, phi, lams, out=out, workspace=ws)
        host.copy_(out, non_blocking=True)
    torch.cuda.synchronize(dev)
    e2e_ms = (time.perf_counter() - t0) * 1e3

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        po = O.ScreenParams(n=1024, pixel_km=float(np.sqrt(lam_ref * O.KM_PER_NM * 160.0 * O.KM_PER_PC / 1024)),
                            r_diff_km=6.0 * pix * np.sqrt(n / 1024), lambda_nm=lam_ref, lambda_ref_nm=lam_ref, seed=7)
        t0 = time.perf_counter()
        O.sum_passband_conjugate(O.make_screen(po), po, lams[::4])
        dt = time.perf_counter() - t0
        cpu = {"value": 1024 * 1024 * len(lams[::4]) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one 1024^2 critical-sampling screen x {len(lams[::4])} wavelengths, {dt:.1f} s"}
    if rank == 0:
        line = {"metric": "one-FFT (Eq. intens) passband pixel-wavelengths/sec at critical sampling",
                "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": f"{count} screens {n}^2, {pix:.2f} km pixels (N Delta^2 = lambda z at 550 nm), "
                                       f"R_diff 3-12 pixels, 32 wavelengths 400-700 nm, patterns resampled onto the "
                                       f"550 nm grid", "l2": "fields of 134 MB per screen and wavelength"},
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": units * world / (e2e_ms * 1e-3), "unit": UNIT,
                        "h2d_bytes_per_step": int(count * (len(lams) * 8 + 96)), "d2h_bytes_per_step": int(count * n * n * 4),
                        "ms_per_step": e2e_ms},
                "transfer_function_same_screens": {"value": units * world / (ms_tf * 1e-3), "ms_per_step": ms_tf},
                "gpu_launches": sum(v["launches"] for v in kstats.values()) * args.steps, "clocks": clk,
                "kernels": {k: {"launches": v["launches"], "ms": v["total_ms"]} for k, v in kstats.items()},
                "kernels_transfer_function": {k: {"launches": v["launches"], "ms": v["total_ms"]}
                                              for k, v in kstats_tf.items()}}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_m_sweep(args):
    """Sect. 4.1 modulation-index sweep through scint_run_batch: R_diff 50..500 km x
    r_s 0.25..1.5 R_sun (Kolmogorov), 8192^2 screens, K_s passband of 21 wavelengths,
    disk, m over the fiducial zone.  Metric: pixel-wavelengths/s."""
    import torch
    import paper_1301_0514_gb300 as S
    import paper_1301_0514_gb300.sweeps as SW

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    pts = SW.sweep_points(n=args.sweep_n, seed=20130514 + 9500 + 100000 * rank)
    lams = SW.KS_BAND_NM
    m = torch.empty((len(pts), 4), dtype=torch.float64, device=dev)
    batch = S.batch_items([dict(params=pt.params, m_map=m[i]) for i, pt in enumerate(pts)])
    ws = torch.empty(S.batch_workspace_bytes(batch, len(lams), args.lanes), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        S.run_batch(batch, lams, n_lanes=args.lanes, workspace=ws)

    step()
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="relaxed"):
        step()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = _max_over_ranks(ms, world, dev)
    units = float(args.sweep_n) ** 2 * len(lams) * len(pts)
    value = units * world / (ms * 1e-3)
    # serial replay for per-kernel times
    S.profile_enable(True)
    pg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(pg, capture_error_mode="relaxed"):
        S.run_batch(batch, lams, n_lanes=1, workspace=ws)
    pg.replay()
    torch.cuda.synchronize(dev)
    kstats = S.profile_read()
    S.profile_enable(False)
    hbm_peak, sm_max_mhz, peak_src = _peaks()
    alu_peak = _sm_count() * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    dom_name, dom = max(kstats.items(), key=lambda kv: kv[1]["total_ms"])
    tflops = dom["flops"] / (dom["total_ms"] * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s", "frac": tflops / alu_peak,
            "traffic": None, "kernel": dom_name, "timing": "serial one-lane replay, CUDA events per launch"}
    mm = m.cpu().numpy()
    rows = SW.summarize(pts, mm[:, 0])
    host = torch.empty((len(pts), 4), dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    step()
    host.copy_(m, non_blocking=True)
    torch.cuda.synchronize(dev)
    e2e_ms = (time.perf_counter() - t0) * 1e3
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        pt = SW.sweep_points(r_diffs=(300.0,), radii_rsun=(0.5,), n=1024, pixels_per_rdiff=0.5)[0]
        po = O.ScreenParams(**pt.params.as_dict())
        t0 = time.perf_counter()
        I = O.smooth_source(O.sum_passband(O.make_screen(po), po, lams), po.pixel_km, po.source_radius_km)
        O.modulation_index_map(I, po)
        dt = time.perf_counter() - t0
        cpu = {"value": 1024 * 1024 * len(lams) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one 1024^2 sweep screen x {len(lams)} wavelengths + disk + m, {dt:.1f} s"}
    if rank == 0:
        line = {"metric": "m-sweep pixel-wavelengths/sec (Sect. 4.1, through scint_run_batch)", "value": value,
                "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic",
                "config": {"workload": f"{len(pts)} Kolmogorov screens {args.sweep_n}^2, R_diff 50..500 km x "
                                       f"r_s 0.25..1.5 R_sun, pixel R_diff/3, z0 160 pc, z1 1 kpc, K_s passband "
                                       f"21 wavelengths, disk, m over the fiducial zone, {args.lanes} lanes",
                           "l2": "fields of 268 MB per screen and wavelength"},
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": units * world / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 21 * 8 + 144 * len(pts),
                        "d2h_bytes_per_step": 32 * len(pts), "ms_per_step": e2e_ms},
                "gpu_launches": sum(v["launches"] for v in kstats.values()) * args.steps, "clocks": clk,
                "xparam": [{"m_theory_bin": r[0], "m_mean": r[1], "m_rms": r[2], "patterns": r[3]} for r in rows],
                "kernels": {k: {"launches": v["launches"], "ms": v["total_ms"]} for k, v in kstats.items()}}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_timeseries(args):
    """Sect. 5 light-curve analysis on one 8192^2 disk-source pattern: curves along
    1024 base tracks and their parallels at 6 separations (0.05..4 R_ref), periodograms
    of every curve, correlation of each base curve with its parallels.
    Metric: curve samples analysed per second."""
    import torch
    import paper_1301_0514_gb300 as S
    import paper_1301_0514_gb300.timeseries as TS

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    n, pix, ns, nb = 8192, 10.0, 4096, 1024
    r_ref = 550.0 * 1e-12 * 160.0 * 3.0856775814913673e13 / 300.0
    p = S.params(n=n, pixel_km=pix, r_diff_km=300.0, lambda_nm=550.0, source_radius_km=0.5 * r_ref,
                 seed=20130514 + 9600 + 100000 * rank)
    I = S.propagate(p, S.make_screen(p))
    S.smooth_source(p, I)
    rng = np.random.default_rng(20130514 + 9601 + rank)
    base = np.stack([rng.uniform(0, n, nb), rng.uniform(0, n, nb), rng.uniform(0, np.pi, nb), np.ones(nb)], axis=1)
    sep = np.array([0.0, 0.05, 0.2, 1.0, 2.5, 4.0]) * r_ref / pix
    tracks = np.concatenate([TS.parallel_tracks(tr, sep) for tr in base], axis=0)
    nc = len(tracks)
    curves = torch.empty((nc, ns), dtype=torch.float32, device=dev)
    power = torch.empty((nc, ns // 2 + 1), dtype=torch.float32, device=dev)
    r = torch.empty((nb, len(sep)), dtype=torch.float64, device=dev)
    ws = torch.empty(8 * ns + 256, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        S.lightcurve(p, I, tracks, ns, out=curves)
        S.curve_power_spectrum(curves, out=power, workspace=ws)
        S.curve_correlation(curves, curves, out=r.view(-1), a_rows=nb, a_stride=len(sep) * ns)

    step()
    torch.cuda.synchronize(dev)
    S.profile_enable(True)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="relaxed"):
        step()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    kstats = S.profile_read()
    S.profile_enable(False)
    ms = e0.elapsed_time(e1) / args.steps
    ms = _max_over_ranks(ms, world, dev)
    units = float(nc) * ns
    value = units * world / (ms * 1e-3)
    hbm_peak, sm_max_mhz, peak_src = _peaks()
    alu_peak = _sm_count() * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    ps = kstats["power_spectrum"]
    tflops = ps["flops"] / (ps["total_ms"] * 1e-3) / 1e12
    gbs = ps["bytes"] / (ps["total_ms"] * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
            "traffic": None, "kernel": "power_spectrum", "fft_tflops": tflops, "alu_frac": tflops / alu_peak,
            "peak_source": f"hbm {peak_src} (MEASURED_PEAKS.json)",
            "note": "per-launch events inside the replayed graph"}
    rm = r.cpu().numpy().mean(axis=0)
    host_r = torch.empty_like(r, device="cpu").pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    step()
    host_r.copy_(r, non_blocking=True)
    torch.cuda.synchronize(dev)
    e2e_ms = (time.perf_counter() - t0) * 1e3
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        hc = curves.cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        O.periodogram(hc)
        for i in range(nb):
            O.pearson(np.repeat(hc[6 * i:6 * i + 1], 6, 0), hc[6 * i:6 * i + 6])
        dt = time.perf_counter() - t0
        cpu = {"value": hc.size / dt, "unit": "curve samples/s", "cores": 1, "kind": "oracle",
               "sample": f"periodograms and correlations of {hc.shape[0]} of the {nc} curves, {dt:.2f} s"}
    if rank == 0:
        line = {"metric": "light-curve samples analysed/sec (Sect. 5: periodograms + two-telescope correlations)",
                "value": value, "unit": "curve samples/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": f"one {n}^2 disk-source pattern (R_diff 300 km, R_s = R_ref/2 at 550 nm), "
                                       f"{nb} tracks x 6 parallels (0..4 R_ref) x {ns} samples",
                           "l2": "curves 100 MB, the map 268 MB"},
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": units * world / (e2e_ms * 1e-3), "unit": "curve samples/s",
                        "h2d_bytes_per_step": int(tracks.nbytes), "d2h_bytes_per_step": int(r.numel() * 8),
                        "ms_per_step": e2e_ms},
                "gpu_launches": sum(v["launches"] for v in kstats.values()) * args.steps, "clocks": clk,
                "mean_correlation_vs_separation_in_R_ref": {f"{d:.2f}": float(v) for d, v in
                                                           zip(sep * pix / r_ref, rm)},
                "kernels": {k: {"launches": v["launches"], "ms": v["total_ms"]} for k, v in kstats.items()}}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_small256(args):
    """The plain method in FP64 (the small-screen configuration): one 256^2 Kolmogorov screen,
    20 km pixels, R_diff 100 km, 500 nm, 160 pc, point source; a step is the synthesis, the FP64
    propagation (scint_propagate64) and the horizontal track through row 128 (integer positions:
    the map's row).  Metric: screen pixels per second.  The oracle does the same in FP64."""
    import torch
    import paper_1301_0514_gb300 as S
    from paper_1301_0514_gb300 import workloads as W

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    it = W.small_screen_256()[0]
    it["seed"] += 100000 * rank
    p = S.params(**{k: it[k] for k in PARAM_KEYS})
    n = p.n
    ws = torch.empty(S.workspace_bytes(p, 1), dtype=torch.uint8, device=dev)
    phi = torch.empty((n, n), dtype=torch.float64, device=dev)
    inten = torch.empty((n, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        S.make_screen(p, out=phi, workspace=ws)
        S.propagate64(p, phi, out=inten, workspace=ws)

    step()
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="relaxed"):
        step()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = _max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    value = float(n) * n * world / (ms * 1e-3)
    # end to end: the call sequence plus the track (row 128) read back to the host each step
    track = torch.empty(n, dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
        track.copy_(inten[128], non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        po = O.ScreenParams(**{k: it[k] for k in PARAM_KEYS})
        reps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < 5.0:
            phi_o = O.make_screen(po)
            I_o = O.intensity_mono(phi_o, po)
            O.lightcurves(I_o, it["tracks"], it["n_samples"])
            reps += 1
        dt = (time.perf_counter() - t0) / reps
        err = float(np.abs(inten.cpu().numpy() - I_o).max())
        cpu = {"value": n * n / dt, "unit": "pixels/s", "cores": 1, "kind": "oracle",
               "sample": f"the whole configuration ({reps} repetitions, {dt * 1e3:.1f} ms each)",
               "gpu_max_abs_err": err}
    if rank == 0:
        print(json.dumps({"metric": "screen pixels propagated per second, FP64 plain method", "value": value,
                          "unit": "pixels/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "one 256^2 Kolmogorov screen, 20 km pixels, R_diff 100 km, 500 nm, "
                                                 "160 pc, point source, taper margin L/4; synthesis + FP64 "
                                                 "propagation (+ the horizontal track in e2e)",
                                     "l2": "inputs fit in L2 (1.5 MB); the configuration is this small"},
                          "e2e": {"value": float(n) * n * world / (e2e_ms * 1e-3), "unit": "pixels/s",
                                  "h2d_bytes_per_step": 0, "d2h_bytes_per_step": n * 8, "ms_per_step": e2e_ms},
                          "gpu_launches": 4 * args.steps, "clocks": clk, "cpu_baseline": cpu}), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_gradient(args):
    """Gradient of a light-curve misfit (the differentiable path): 8 screens of 2048^2,
    R_diff 100 km, 500 nm, one track of 10^4 samples at 0.2 px per screen.  A step is the
    forward pass (screen -> propagation -> curve) and the adjoint (dL/dphi, dL/dR_diff)
    for every screen.  Metric: screen pixels differentiated per second."""
    import torch
    import paper_1301_0514_gb300 as S
    from paper_1301_0514_gb300 import workloads as W

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    items = W.gradient_batch_2048()
    for it in items:
        it["seed"] += 100000 * rank
    P = [S.params(**{k: it[k] for k in PARAM_KEYS}) for it in items]
    n = items[0]["n"]
    lams = items[0]["lambdas_nm"]
    ws = torch.empty(S.workspace_bytes(P[0], len(lams)), dtype=torch.uint8, device=dev)
    phi = [torch.empty((n, n), dtype=torch.float64, device=dev) for _ in items]
    inten = torch.empty((n, n), dtype=torch.float32, device=dev)
    curves = [torch.empty((1, it["n_samples"]), dtype=torch.float32, device=dev) for it in items]
    targets = [torch.rand((1, it["n_samples"]), generator=torch.Generator().manual_seed(7 + i)).to(dev)
               for i, it in enumerate(items)]
    gcur = [torch.empty_like(c) for c in curves]
    gphi = [torch.empty((n, n), dtype=torch.float64, device=dev) for _ in items]
    grd = [torch.empty(1, dtype=torch.float64, device=dev) for _ in items]
    for p, f in zip(P, phi):
        S.make_screen(p, out=f, workspace=ws)
    stream = torch.cuda.current_stream(dev)

    def step():
        for i, (p, it) in enumerate(zip(P, items)):
            S.sum_passband(p, phi[i], lams, out=inten, workspace=ws)
            S.lightcurve(p, inten, it["tracks"], it["n_samples"], out=curves[i])
            torch.sub(curves[i], targets[i], out=gcur[i])          # dL/dc of L = sum (c - t)^2 / 2
            S.lightcurve_adjoint(p, phi[i], lams, it["tracks"], it["n_samples"], gcur[i], out=gphi[i],
                                 workspace=ws)
            S.rdiff_gradient(p, phi[i], gphi[i], workspace=ws, out=grd[i])

    step()
    torch.cuda.synchronize(dev)
    S.profile_enable(True)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="relaxed"):
        step()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    kstats = S.profile_read()
    S.profile_enable(False)
    ms = _max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    units = float(n) * n * len(items)
    value = units * world / (ms * 1e-3)
    hbm_peak, sm_max_mhz, peak_src = _peaks()
    alu_peak = _sm_count() * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    dom_name, dom = max(kstats.items(), key=lambda kv: kv[1]["total_ms"])
    tflops = dom["flops"] / (dom["total_ms"] * 1e-3) / 1e12 if dom["flops"] else 0.0
    gbs = dom["bytes"] / (dom["total_ms"] * 1e-3) / 1e9
    roof = ({"bound": "alu", "achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s", "frac": tflops / alu_peak}
            if dom["flops"] else {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak})
    roof.update({"traffic": None, "kernel": dom_name, "share": dom["total_ms"] / ms,
                 "timing": "per-launch events inside the replayed graph"})
    host = torch.empty(len(items), dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    step()
    host.copy_(torch.cat(grd), non_blocking=True)
    torch.cuda.synchronize(dev)
    e2e_ms = (time.perf_counter() - t0) * 1e3
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        it = dict(items[0])
        po = O.ScreenParams(**{k: it[k] for k in PARAM_KEYS}).with_(n=1024)
        phi_o = O.make_screen(po)
        tgt = np.zeros((1, it["n_samples"]))
        tr = np.array(it["tracks"], dtype=np.float64).reshape(-1, 4).copy()
        tr[:, [0, 1, 3]] *= 0.5                   # the same track on a half-size grid
        t0 = time.perf_counter()
        O.misfit_gradient(po, phi_o, lams, tr, it["n_samples"], tgt)
        dt = time.perf_counter() - t0
        cpu = {"value": 1024 * 1024 / dt, "unit": "screen pixels/s", "cores": 1, "kind": "oracle",
               "sample": f"one 1024^2 screen, forward + adjoint, {dt:.1f} s"}
    if rank == 0:
        line = {"metric": "screen pixels differentiated/sec (forward + adjoint of a light-curve misfit)",
                "value": value, "unit": "screen pixels/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": f"{len(items)} screens {n}^2, 10 km pixels, R_diff 100 km, 500 nm, one track of "
                                       f"10^4 samples at 0.2 px; forward + dL/dphi + dL/dR_diff per screen",
                           "l2": "fields of 34 MB per screen"},
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": units * world / (e2e_ms * 1e-3), "unit": "screen pixels/s",
                        "h2d_bytes_per_step": int(len(items) * (32 + 8 + 96)), "d2h_bytes_per_step": 8 * len(items),
                        "ms_per_step": e2e_ms},
                "gpu_launches": sum(v["launches"] for v in kstats.values()) * args.steps, "clocks": clk,
                "kernels": {k: {"launches": v["launches"], "ms": v["total_ms"]} for k, v in kstats.items()}}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch-mode", default="tune", choices=["tune", "lanes", "persistent"],
                    help="batch form: chosen by the batch tuner, or fixed")
    ap.add_argument("--plans", default="tune", choices=["tune", "unpacked", "packed"],
                    help="propagation plans: autotuned per grid size, or fixed")
    ap.add_argument("--workload", default="batched", choices=["batched", "single4096", "profile", "large16384", "screen_check", "conjugate",
                                                              "m_sweep", "timeseries", "gradient", "small256"])
    ap.add_argument("--profile-screens", type=int, default=1, help="4096^2 screens of the profile workload (1..16)")
    ap.add_argument("--check-n", type=int, default=14000, help="grid of the screen-check workload")
    ap.add_argument("--conj-n", type=int, default=4096, help="grid of the one-FFT workload")
    ap.add_argument("--sweep-n", type=int, default=8192, help="grid of the m-sweep workload")
    ap.add_argument("--lanes", type=int, default=8, help="streams the batch is scheduled on (1..8)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.workload == "screen_check" and args.impl != "reference":
        run_screen_check(args)
    elif args.workload == "conjugate" and args.impl != "reference":
        run_conjugate(args)
    elif args.workload == "m_sweep" and args.impl != "reference":
        run_m_sweep(args)
    elif args.workload == "timeseries" and args.impl != "reference":
        run_timeseries(args)
    elif args.workload == "small256" and args.impl != "reference":
        run_small256(args)
    elif args.workload == "gradient" and args.impl != "reference":
        run_gradient(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
