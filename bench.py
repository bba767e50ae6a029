#!/usr/bin/env python
"""Benchmark of the GB300 3D MOC transport sweep.

Metric: 3D MOC segment-group integrations per second (one integration = Eq. 3
on one 3D segment, in one direction, for one energy group, plus its Eq. 4
tally).  Workload: the 17x17 pin lattice (synthetic, seeded; 7 groups, 32
azimuths x 4 polar angles, 0.05 cm radial and 0.5 cm axial spacing, 20 cm in
10 layers, reflective radially, vacuum axially), FP32 sweep, all segment
templates stored.  A step is one outer power iteration on the device-resident
problem: source update, sweep, flux / k / residual update.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  With --impl reference the FP64 CPU oracle runs the
same steps on the host cores (rank 0 only).
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "3D MOC segment-group integrations/s"
UNIT = "integrations/s"
WORKLOAD = "lattice17"
WORKLOAD_DESC = ("17x17 pin lattice (264 fuel pins, 25 seeded guide tubes), 3 materials, 7 groups, "
                 "20 cm in 10 layers, reflective radial / vacuum axial, 32 azimuthal x 4 polar, "
                 "radial spacing 0.05 cm, axial spacing 0.5 cm; FP32 sweep, templates stored")
# algorithmic work of one integration: 7 FP32 operations, one of them the exponential
OPS_PER_INTEGRATION = 7
# shared-memory bytes of one integration in the privatised-tally design: Qr and
# Sigma_t of the FSR-group (4 + 4) and the tally word (4)
SMEM_BYTES_PER_INTEGRATION = 12
# ALU roofline: the FP32 lane-operation rate MEASURED on the device at the
# start of the run (moc_measure_unit_rates: fused multiply-adds, scalar and as
# packed pairs, every SM filled); the SM count is the device's.  The
# exponential unit (moc_measure_ex2_rate, ~31 ex2 per SM per clock) would
# allow 1.4x more integrations per second than the FP32 pipe, so it does not bind.
# FP64 sweeps are bound by the FP64 pipe: 2 lane operations per SM per clock
# (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on peak_sustained).  Each
# integration takes 15 FP64 operations as written: Sigma_t l (1), the
# table-driven e^{-x} (11), d = psi - W S Qr, d (1 - e), psi -= (3)
SM_MAX_MHZ = 2070.0
FP64_LANES_PER_CLK, FP64_OPS_PER_INTEGRATION = 2, 15
STEP_DESC = "one outer power iteration: source, sweep, flux/k/residual update"
L2_FLUSH_BYTES = 256 << 20


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def whole_job_rate(local_seconds, units_per_rank, world, device=None):
    """Whole-job rate of weakly scaled replicas: every rank processed
    units_per_rank units in local_seconds; the job's time is the slowest
    rank's (an all-reduce MAX over the default process group when world > 1).
    Returns (units per second over all ranks, job seconds)."""
    total_s = float(local_seconds)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    return world * units_per_rank / total_s, total_s


def clock_sampler(device, path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", f"--id={device}", f"--query-gpu={q}",
                                 "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def parse_clocks(path):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
    except OSError:
        pass
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def profile_traffic(src_hash):
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on the current sweep source; otherwise None."""
    path = os.path.join(ROOT, "profiles", "k_sweep_lattice17.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9]+)", txt)
    if not m or not t or m.group(1) != src_hash:
        return None
    return int(t.group(1))


def measured_hbm_gbs():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return None


def sweep_source_hash():
    h = hashlib.sha256()
    for f in ("moc_sweep_kernel.cuh", "moc_device.cuh", "moc_exp64.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2503_17743_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def cpu_baseline(prob, seconds_target=10.0):
    """The oracle (as it stands) on the host cores: full FP64 sweeps of the
    workload from a seeded source, as many as fit in about 10 s; then on one
    thread, the 2D tracks of one sweep in index order for about 5 s."""
    import numpy as np

    import oracle
    cores = os.cpu_count() or 1
    o = oracle.Oracle(prob, n_threads=cores)
    Q = np.random.default_rng(7).uniform(0.2, 1.0, size=(o.n_fsr, prob.num_groups))
    n_total, t_total, sweeps = 0, 0.0, 0
    while t_total < seconds_target and sweeps < 20:
        t0 = time.perf_counter()
        n, _ = o.sweep_sample(Q, 0, o.n_tracks2d)
        t_total += time.perf_counter() - t0
        n_total += n
        sweeps += 1
    o.set_threads(1)
    n1, t1, t = 0, 0.0, 0
    step = max(1, o.n_tracks2d // 32)
    while t1 < seconds_target / 2 and t < o.n_tracks2d:
        t_end = min(t + step, o.n_tracks2d)
        t0 = time.perf_counter()
        n, _ = o.sweep_sample(Q, t, t_end)
        t1 += time.perf_counter() - t0
        n1 += n
        t = t_end
    return {"value": n_total / t_total, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{sweeps} full FP64 sweep(s) of {WORKLOAD} from a seeded source "
                      f"({n_total:.4g} integrations, {t_total:.1f} s)",
            "single_thread": {"value": n1 / t1, "unit": UNIT, "cores": 1,
                              "sample": f"2D tracks 0-{t} of {o.n_tracks2d} of one sweep "
                                        f"({n1:.4g} integrations, {t1:.1f} s)"}}


def bench_config():
    """The `config` of both arms' lines: the workload and the step (the same
    keys and values, so that the two lines are like for like)."""
    return {"workload": WORKLOAD_DESC, "step": STEP_DESC}


def run_reference(args):
    import synth
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    prob = synth.workload(WORKLOAD)
    cores = os.cpu_count() or 1
    o = oracle.Oracle(prob, n_threads=cores)
    o.reset()
    integ_per_step = None
    for _ in range(args.warmup):
        o.iterate(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.iterate(1)
    dt = time.perf_counter() - t0
    # integrations of one sweep (the oracle counts them in a sample sweep)
    import numpy as np
    n, _ = o.sweep_sample(np.zeros((o.n_fsr, prob.num_groups)), 0, o.n_tracks2d)
    integ_per_step = n
    value = integ_per_step * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": bench_config(),
            "details": {"arm": "FP64 oracle on the host cores, as it stands"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} outer iterations of {WORKLOAD}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    import synth
    from paper_2503_17743_gb300 import MOC_FP32, Geometry, Tracks, load, track_params
    from paper_2503_17743_gb300 import build as libbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    libbuild.build()
    load()
    # the device's unit rates (FP32 pipe, shared memory): the roofline peaks
    from paper_2503_17743_gb300 import measure_unit_rates
    rates = measure_unit_rates(local)
    prob = synth.workload(WORKLOAD)
    geom = Geometry(prob)
    params = track_params(prob, precision=MOC_FP32, device=local)
    schedule = None
    if args.tune:
        # the launch schedule (groups per lane, tally mode, preload split) from
        # the project's autotuner; every candidate is timed outside the
        # measured region
        from paper_2503_17743_gb300 import autotune
        params, t_best, table = autotune(geom, params, iterations=5)
        schedule = {"groups_per_lane": params.groups_per_lane, "tally_mode": params.tally_mode,
                    "preload_budget_bytes": params.preload_budget_bytes, "sync_block": params.sync_block,
                    "tuned_ms_per_iteration": t_best * 1e3,
                    "candidates": [[int(r[0]), int(r[1]), int(r[2]), int(r[5]), round(r[4] * 1e3, 4)]
                                   for r in table],
                    "candidate_columns": ["groups_per_lane", "tally_mode", "preload_budget", "sync_block",
                                          "ms_per_iteration"]}
    tr = Tracks(geom, params)
    info = tr.info
    integ = info["integrations_per_sweep"]
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        tr.enqueue_source(sp)
        ev_s0.record(stream)
        tr.enqueue_sweep(sp)
        ev_s1.record(stream)
        tr.enqueue_update(sp)

    # warm-up (also warms the kernels' first-launch costs)
    tr.reset()
    ev_s0, ev_s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 0)):
            step()
    torch.cuda.synchronize()

    steps = []
    for _ in range(args.steps):
        steps.append([torch.cuda.Event(enable_timing=True) for _ in range(4)])
    sampler, clk_file = (None, None)
    clk_path = os.path.join(tempfile.gettempdir(), f"moc_bench_clocks_{os.getpid()}_{rank}.csv")
    if rank == 0:
        sampler, clk_file = clock_sampler(local, clk_path)
        time.sleep(0.5)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for evs in steps:
            flush.zero_()                 # L2 flushed between timed steps, outside the events
            evs[0].record(stream)
            tr.enqueue_source(sp)
            evs[1].record(stream)
            tr.enqueue_sweep(sp)
            evs[2].record(stream)
            tr.enqueue_update(sp)
            evs[3].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    if sampler is not None:
        sampler.terminate()
        sampler.wait()
        clk_file.close()
    step_ms = [e[0].elapsed_time(e[3]) for e in steps]
    sweep_ms = [e[1].elapsed_time(e[2]) for e in steps]
    res = tr.read_result(sp)
    value, total_s = whole_job_rate(sum(step_ms) * 1e-3, integ * args.steps, world, device="cuda")

    # end to end through the C ABI from host arrays: geometry, tracks, a
    # converged eigenvalue solve, the flux read back
    e2e = None
    if rank == 0:
        e2e_runs = []
        for _ in range(max(1, min(args.steps, args.e2e_runs))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g2 = Geometry(prob)
            t2 = Tracks(g2, params)
            r2 = t2.solve_eigen(tol_k=1e-7, tol_src=1e-6, max_iter=5000, use_graph=True, check=False)
            phi, k2 = t2.flux()
            dt = time.perf_counter() - t0
            h2d = t2.info.get("h2d_bytes", 0)
            t2.close()
            e2e_runs.append((r2["integrations"] / dt, dt, r2, h2d, phi.nbytes + 128 * r2["iterations"], k2))
        best = max(e2e_runs, key=lambda x: x[0])
        e2e = {"value": best[0], "unit": UNIT, "h2d_bytes_per_step": int(best[3]),
               "d2h_bytes_per_step": int(best[4]), "seconds": best[1],
               "iterations": best[2]["iterations"], "k": best[5],
               "step": "moc_create_geometry + moc_generate_tracks + moc_solve_eigen "
                       "(tol_k 1e-7, tol_src 1e-6, CUDA graphs) + moc_get_flux, from host arrays"}
        gk = golden_k()
        if gk is not None:
            e2e["k_oracle"] = gk
            e2e["k_err"] = abs(best[5] - gk)

    if rank != 0:
        return
    sw = statistics.mean(sweep_ms) * 1e-3
    roof = alu_roofline(integ, sw, rates)
    traffic = profile_traffic(sweep_source_hash())
    roof["traffic"] = traffic
    # the HBM side of the same sweep: algorithmic bytes (boundary fluxes in
    # and out, stored template records) and, from the committed ncu summary,
    # the DRAM bytes moved, both per launch time, against the measured copy peak
    alg_bytes = 2 * (info["tracks3d"] // 2) * 4 * prob.num_groups * 4 + info["stored_segments"] * 8
    hbm_peak = measured_hbm_gbs()
    roof["hbm"] = {"algorithmic_bytes": alg_bytes, "algorithmic_gbs": alg_bytes / sw / 1e9,
                   "dram_gbs": traffic / sw / 1e9 if traffic else None,
                   "peak_gbs": hbm_peak,
                   "frac": (traffic / sw / 1e9) / hbm_peak if (traffic and hbm_peak) else None}
    clocks = parse_clocks(clk_path)
    try:
        os.remove(clk_path)
    except OSError:
        pass
    cpu = cpu_baseline(prob) if (world == 1 and not args.no_cpu_baseline) else None
    # the same workload with FP64 sweeps (parity precision), device-resident
    fp64 = None
    if rank == 0 and args.fp64_steps > 0:
        from paper_2503_17743_gb300 import MOC_FP64, autotune
        p64 = track_params(prob, precision=MOC_FP64, device=local)
        sched64 = None
        if args.tune:
            p64, t64_best, _ = autotune(geom, p64, iterations=3)
            sched64 = {"tally_mode": int(p64.tally_mode), "preload_budget_bytes": int(p64.preload_budget_bytes),
                       "tuned_ms_per_iteration": t64_best * 1e3}
        t64 = Tracks(geom, p64)
        t64.iterate(3, use_graph=True)
        r64 = t64.iterate(args.fp64_steps, use_graph=True)
        rate64 = r64["integrations"] / r64["seconds"]
        peak64 = rates["sm_count"] * FP64_LANES_PER_CLK * SM_MAX_MHZ * 1e6 / 1e12
        fp64 = {"value": rate64, "unit": UNIT,
                "ms_per_step": r64["seconds"] / args.fp64_steps * 1e3, "steps": args.fp64_steps,
                "dtype": "f64", "timing": "CUDA events around the graph launches of the steps",
                "schedule": sched64,
                "roofline": {"bound": "alu", "achieved": rate64 * FP64_OPS_PER_INTEGRATION / 1e12,
                             "peak": peak64, "unit": "TFLOP/s",
                             "frac": rate64 * FP64_OPS_PER_INTEGRATION / 1e12 / peak64,
                             "peak_basis": f"derived: FP64 pipe 2 lane operations per SM per clock x "
                                           f"{rates['sm_count']} SMs x 2070 MHz; 15 FP64 operations per "
                                           "integration (whole step timed: the sweep is most of it)"}}
        t64.close()
    tr.close()
    ablation = run_ablation_rows(WORKLOAD, local) if (rank == 0 and args.ablation_leg) else None
    large = None
    if rank == 0 and args.large:
        large = [run_large(name, local, rates, oracle_seconds=args.large_oracle_seconds)
                 for name in ("asm3x3", "core7x7")]
    serving = None
    if rank == 0 and args.serving_requests > 0:
        serving = run_serving_rates(args.serving_requests, device=local,
                                    load_factors=tuple(float(x) for x in args.serving_loads.split(",")))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_s / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": bench_config(),
            "details": {"parallelism": f"replicas x{world}",
                        "integrations_per_step": integ, "segments3d": info["segments3d"],
                        "l2": "flushed between timed steps (256 MiB write outside the events)",
                        "k_after_steps": res["k"], "schedule": schedule,
                        "sync_block": info.get("sync_block"), "tally_bits": info.get("tally_bits"),
                        "unit_rates": rates},
            "roofline": roof, "clocks": clocks, "cpu_baseline": cpu, "e2e": e2e, "fp64": fp64,
            "large": large, "serving": serving, "ablation": ablation,
            "gpu_launches": 6 * args.steps}
    print(json.dumps(line), flush=True)


def alu_roofline(integrations, sweep_s, rates):
    """Roofline of one sweep launch against the device's MEASURED FP32 rate
    (7 FP32 operations per integration), with the shared-memory side of the
    same launch (12 algorithmic bytes per integration against the measured
    conflict-free shared-memory load rate)."""
    peak_ops = max(rates["fp32_fma_scalar_per_s"], rates["fp32_fma_packed_lane_ops_per_s"])
    ach = OPS_PER_INTEGRATION * integrations / sweep_s / 1e12
    peak = peak_ops / 1e12
    smem_peak = rates["smem_load_bytes_per_s"] / 1e9
    smem_ach = SMEM_BYTES_PER_INTEGRATION * integrations / sweep_s / 1e9
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "kernel": "k_sweep", "sweep_ms": sweep_s * 1e3,
            "peak_basis": f"of measured: FP32 lane operations per second on this device "
                          f"(moc_measure_unit_rates, {rates['sm_count']} SMs at {rates['sm_mhz']:.0f} MHz; "
                          "scalar and packed f32x2 FMAs measure the same rate); "
                          "7 FP32 operations per integration",
            "smem": {"algorithmic_bytes_per_integration": SMEM_BYTES_PER_INTEGRATION,
                     "achieved_gbs": smem_ach, "peak_gbs": smem_peak, "frac": smem_ach / smem_peak,
                     "peak_basis": "of measured: conflict-free 16-byte shared-memory loads"}}


def run_large(name, device, rates, iters=3, oracle_seconds=6.0):
    """One of the large configurations (3x3 assemblies + reflector, 64 cm,
    64 x 6 directions, a preload budget below the full template set; the 7x7
    core with a reflector ring, 200 cm, 128 x 6, all vacuum), FP32: track
    generation, one warm-up and `iters` graph-launched outer iterations timed
    with CUDA events, clocks sampled during them; the roofline against the
    same measured FP32 peak; the FP64 oracle on the host cores timed on a
    sample of 2D tracks of one sweep and extrapolated (labelled as such)."""
    import numpy as np

    import oracle
    import synth
    from paper_2503_17743_gb300 import MOC_FP32, Geometry, Tracks, track_params
    p = synth.workload(name)
    budget = (1 << 30) if name == "asm3x3" else -1
    t0 = time.perf_counter()
    tr = Tracks(Geometry(p), track_params(p, precision=MOC_FP32, device=device,
                                          preload_budget_bytes=budget, trace_on_device=1))
    gen_s = time.perf_counter() - t0
    info = tr.info
    tr.iterate(1, use_graph=True)
    clk_path = os.path.join(tempfile.gettempdir(), f"moc_large_clocks_{os.getpid()}.csv")
    sampler, clk_file = clock_sampler(device, clk_path)
    time.sleep(0.3)
    r = tr.iterate(iters, use_graph=True)
    if sampler is not None:
        sampler.terminate()
        sampler.wait()
        clk_file.close()
    clocks = parse_clocks(clk_path)
    try:
        os.remove(clk_path)
    except OSError:
        pass
    rate = r["integrations"] / r["seconds"]
    integ = info["integrations_per_sweep"]
    tr.close()
    # the oracle on a sample: 2D tracks from four places of the laydown
    o = oracle.Oracle(p, n_threads=os.cpu_count() or 1, light=True)
    Q = np.random.default_rng(3).uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    n_s, t_s, tracks = 0, 0.0, 0
    k = max(1, o.n_tracks2d // 400)
    for frac in (0.125, 0.375, 0.625, 0.875, 0.0625, 0.3125, 0.5625, 0.8125):
        a = int(frac * o.n_tracks2d)
        t1 = time.perf_counter()
        n, _ = o.sweep_sample(Q, a, min(a + k, o.n_tracks2d))
        t_s += time.perf_counter() - t1
        n_s += n
        tracks += min(a + k, o.n_tracks2d) - a
        if t_s > oracle_seconds:
            break
    del o
    roof = alu_roofline(integ, r["seconds"] / iters, rates)
    roof["sweep_ms"] = None
    roof["timing"] = "whole outer iteration (the sweep is nearly all of it)"
    return {"workload": name, "integrations_per_sweep": integ, "value": rate, "unit": UNIT,
            "ms_per_iteration": r["seconds"] / iters * 1e3, "iterations": iters,
            "generation_s": gen_s, "preloaded_stacks": info["preloaded_stacks"], "stacks": info["stacks"],
            "stored_segments": info["stored_segments"], "chunk_segments": info["chunk_segments"],
            "tally_bits": info.get("tally_bits"),
            "device_bytes": info["device_bytes"], "clocks": clocks, "roofline": roof,
            "cpu_baseline": {"value": n_s / t_s, "unit": UNIT, "cores": os.cpu_count() or 1,
                             "kind": "oracle",
                             "sample": f"extrapolated: {tracks} of {p.name}'s 2D tracks of one FP64 sweep "
                                       f"({n_s:.4g} integrations, {t_s:.1f} s); a full sweep would take "
                                       f"about {integ / (n_s / t_s):.0f} s"}}


def run_serving_rates(n_requests, device=0, load_factors=(0.5, 1.0, 2.0), seed=1):
    """The serving stream at several arrival rates: the requests solved one at
    a time once (the sequential rate R), then arriving as a Poisson process at
    each load factor x R into the serving engine."""
    seq = sequential_solves(n_requests, device, seed)
    rows = [run_serving(n_requests, seed=seed, load_factor=lf, device=device, seq=seq)
            for lf in load_factors]
    return {"requests": n_requests, "sequential_solves_per_s": seq[0], "rates": rows}


def run_ablation_rows(workload, device):
    """The ablation table (see run_ablation) as a list of rows."""
    class A:
        pass
    a = A()
    a.workload = workload
    a.device = device
    return run_ablation(a, emit=False)


def run_profile_driver(args):
    """Untimed driver for ncu captures: builds the workload's tracks, runs 3
    outer iterations, then 2 more (the 4th and 5th sweeps are the ones a
    capture with -s 3 selects)."""
    import synth
    from paper_2503_17743_gb300 import MOC_FP32, MOC_FP64, Geometry, Tracks, track_params
    prob = synth.workload(args.workload)
    tr = Tracks(Geometry(prob), track_params(prob, preload_budget_bytes=args.budget,
                                             groups_per_lane=args.gpl,
                                             chunk_segments=args.chunk, sync_block=args.sync,
                                             precision=MOC_FP64 if args.fp64 else MOC_FP32))
    tr.iterate(3, use_graph=False)
    r = tr.iterate(2, use_graph=False)
    print(json.dumps({"info": tr.info, "ms_per_iteration": r["seconds"] * 1e3 / 2}), flush=True)
    tr.close()


SERVE_TOL = dict(tol_k=1e-7, tol_src=1e-6, max_iter=4000)


def sequential_solves(n_requests, device=0, seed=1):
    """Every request of the serving stream solved one at a time, end to end
    through the C ABI: (solves per second, k of each, flux of each)."""
    import synth
    from paper_2503_17743_gb300 import Geometry, Tracks, track_params
    probs = [synth.serving_request(seed, i) for i in range(n_requests)]
    t0 = time.perf_counter()
    ks, phis = [], []
    for p in probs:
        tr = Tracks(Geometry(p), track_params(p, device=device))
        if p.ext_source is None:
            r = tr.solve_eigen(**SERVE_TOL)
        else:
            r = tr.solve_fixed_source(tol_src=SERVE_TOL["tol_src"], max_iter=SERVE_TOL["max_iter"])
        phi, _ = tr.flux()
        ks.append(r["k"])
        phis.append(phi)
        tr.close()
    return n_requests / (time.perf_counter() - t0), ks, phis


def run_serving(n_requests, seed=1, load_factor=2.0, device=0, seq=None):
    """Serving stream (seeded serving_request mix: n x n lattices, 2-7 groups,
    2-20 cm, 16-64 azimuths x 2-4 polar, half eigenvalue, half fixed source).
    First every request is solved one at a time in arrival order (sequential
    rate R, unless `seq` gives it); then the same requests arrive as a
    Poisson process at load_factor x R into the serving engine.  Latency =
    completion time minus scheduled arrival time."""
    import numpy as np

    import synth
    from paper_2503_17743_gb300 import Geometry, Server, track_params
    probs = [synth.serving_request(seed, i) for i in range(n_requests)]
    if seq is None:
        seq = sequential_solves(n_requests, device, seed)
    rate_seq, ks, phis = seq
    # batched: Poisson arrivals into the engine
    rng = np.random.default_rng(seed + 1000)
    arrivals = np.cumsum(rng.exponential(1.0 / (load_factor * rate_seq), size=n_requests))
    srv = Server(device=device)
    geoms, tickets, done = {}, {}, {}
    t0 = time.perf_counter()
    nxt = 0
    while len(done) < n_requests:
        now = time.perf_counter() - t0
        while nxt < n_requests and arrivals[nxt] <= now:
            p = probs[nxt]
            geoms[nxt] = Geometry(p)
            tickets[nxt] = srv.submit(geoms[nxt], track_params(p, device=device), **SERVE_TOL)
            nxt += 1
        if len(tickets) > len(done):
            srv.step()
            for i, t in tickets.items():
                if i not in done:
                    r = srv.result(t)
                    if r is not None:
                        done[i] = (time.perf_counter() - t0, r)
                        del geoms[i]
        elif nxt < n_requests:
            time.sleep(max(0.0, min(0.002, arrivals[nxt] - (time.perf_counter() - t0))))
    t_end = max(v[0] for v in done.values())
    lat = np.array([done[i][0] - arrivals[i] for i in range(n_requests)])
    kerr = max(abs(done[i][1][0]["k"] - ks[i]) for i in range(n_requests))
    ferr = max(float(np.max(np.abs(done[i][1][1] - phis[i]) / np.maximum(np.abs(phis[i]), 1e-300)))
               for i in range(n_requests))
    st = srv.stats()
    srv.close()
    return {"requests": n_requests, "load_factor": load_factor,
            "sequential_solves_per_s": rate_seq, "solves_per_s": n_requests / (t_end - arrivals[0]),
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "max_resident": st["max_resident"], "max_k_diff_vs_sequential": kerr,
            "max_flux_rel_diff_vs_sequential": ferr,
            "tolerance": "tol_k 1e-7, tol_src 1e-6, FP32 sweeps",
            "workload": f"seeded serving_request mix, seed {seed}: n x n pin lattices (n 1-17), 2-7 groups, "
                        "2-20 cm, 16-64 azimuths x 2-4 polar, half eigenvalue / half fixed source, "
                        "Poisson arrivals at load_factor x the sequential rate"}


def run_ablation(args, emit=True):
    """The paper's two optimisations measured on this sweep (Sec. 4.2, 4.3;
    Figs. 6 and 7): the stored (EXP) share of the segment templates from 0 to
    100%, and load balancing off (work units and tracks in index order) or on.
    Each line: mean outer-iteration time of 10 graph-launched iterations after
    3 warm-up ones; one JSON line with the table."""
    import synth
    from paper_2503_17743_gb300 import (MOC_SCHED_TRACKS_NATURAL, MOC_SCHED_UNITS_NATURAL, Geometry,
                                        Tracks, track_params)
    prob = synth.workload(args.workload)
    geom = Geometry(prob)
    dev = getattr(args, "device", 0)
    full = Tracks(geom, track_params(prob, preload_budget_bytes=-1, device=dev))
    tpl_bytes = full.info["stored_segments"] * 8
    full.close()
    rows = []

    def measure(label, **kw):
        tr = Tracks(geom, track_params(prob, device=dev, **kw))
        tr.iterate(3, use_graph=True)
        r = tr.iterate(10, use_graph=True)
        info = tr.info
        rows.append({"case": label, "ms_per_iteration": r["seconds"] * 100.0,
                     "integrations_per_s": r["integrations"] / r["seconds"],
                     "stored_segments": info["stored_segments"],
                     "preloaded_stacks": info["preloaded_stacks"], "stacks": info["stacks"]})
        tr.close()

    for frac in (0.0, 0.25, 0.5, 0.75, 1.0):
        measure(f"EXP share {frac:.2f}", preload_budget_bytes=int(frac * tpl_bytes) if frac < 1 else -1)
    measure("load balancing off (units and tracks in index order)",
            schedule=MOC_SCHED_UNITS_NATURAL | MOC_SCHED_TRACKS_NATURAL)
    measure("units largest first, tracks in index order", schedule=MOC_SCHED_TRACKS_NATURAL)
    measure("units in index order, tracks by segment count", schedule=MOC_SCHED_UNITS_NATURAL)
    measure("load balancing on (default)")
    measure("synchronous blocks off (each track on its own records)", sync_block=1)
    if emit:
        print(json.dumps({"ablation": args.workload, "rows": rows}), flush=True)
    return rows


def golden_k():
    path = os.path.join(ROOT, "tests", "golden", "oracle_k.json")
    try:
        return json.load(open(path))[WORKLOAD]["k"]
    except (OSError, KeyError, ValueError):
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-runs", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=5, help="timed FP64 steps (0 = skip)")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="skip the schedule autotuner (default parameters)")
    ap.add_argument("--serving-requests", type=int, default=256,
                    help="requests of the serving leg (0 = skip)")
    ap.add_argument("--serving-loads", default="0.5,1,2",
                    help="arrival rates of the serving leg, as multiples of the sequential rate")
    ap.add_argument("--no-large", dest="large", action="store_false",
                    help="skip the large-configuration leg (3x3 assemblies, 7x7 core)")
    ap.add_argument("--large-oracle-seconds", type=float, default=6.0,
                    help="host-core seconds of the oracle sample per large configuration")
    ap.add_argument("--no-ablation-leg", dest="ablation_leg", action="store_false",
                    help="skip the ablation table in the bench line")
    ap.add_argument("--ablation", action="store_true",
                    help="EXP share and load-balancing ablation table (JSON)")
    ap.add_argument("--profile", action="store_true",
                    help="untimed 3 + 2 iterations (driver of the ncu captures)")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--budget", type=int, default=-1, help="preload budget bytes (--profile)")
    ap.add_argument("--gpl", type=int, default=0, help="groups per lane (--profile)")
    ap.add_argument("--fp64", action="store_true", help="FP64 sweeps (--profile)")
    ap.add_argument("--chunk", type=int, default=0,
                    help="2D segments per radial chunk, 0 = automatic (--profile)")
    ap.add_argument("--sync", type=int, default=0,
                    help="tracks per synchronous block, 0 = default (--profile)")
    args = ap.parse_args()
    if args.profile:
        run_profile_driver(args)
        return
    if args.ablation:
        run_ablation(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
