#!/usr/bin/env python3
"""Benchmark of the Shan-Chen bubble-merging LBM hot path on GB300.

One bench step = one diagnostic interval of the 512^3 D3Q19 FP32 foam
workload (1000 seeded gas bubbles, radii uniform 4..12, tau 0.8, G -5): 100
fused collide-stream-force steps, then the diagnostics of the interval: FP64
totals and gas labelling in one pass, the per-site merge bookkeeping, the
FP64 EOS pressure and the film test at every lattice point, and the bubble
census with its size histogram, all through the C ABI.  Throughput is
MLUPS = cells * 100 / seconds / 1e6 over the whole step.  The default 20
timed bench steps cover the workload's 2000 LBM steps.  --workload foam128
(64 injecting nuclei on 128^3), foam768 (the FP16 full foam) and ensemble256
(the batched two-bubble sweep) select the other workloads; --storage
f16/bf16/f64 the storage form.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 is launched with torch.distributed.run: every rank advances its own
replica of the lattice (the workload has no exchange step between
independent lattices), the timed region is bracketed by barriers and the
maximum time over ranks is reported.  --impl reference times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1708_01608_gb300.workloads import FOAM_512 as W  # noqa: E402

METRIC = ("D3Q19 Shan-Chen MLUPS (512^3 foam, FP32 storage, 1000 bubbles, "
          "diagnostics every 100 steps)")
UNIT = "MLUPS"
INNER = 100                                   # LBM steps per bench step
CELLS = W["nx"] * W["ny"] * W["nz"]
Q = 19
B_ALG = 2 * Q * 4                             # bytes per lattice update, FP32 storage
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes per launch of the fused kernel (dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture of the current kernel), keyed by
# (workload, storage, tile id); workloads without a capture of the current
# kernel report null.  The 512^3 entries are the 256^3 capture of the same
# tile scaled by the cells per launch (x8): at 256^3 the lattice is already
# five times the L2 and the capture's traffic equals the algorithmic bytes.
NCU_TRAFFIC_PER_LAUNCH = {("d3q19_foam_128", "f32", 25): 277.73e6,
                          ("d3q19_foam_128", "f64", 6): 626.48e6,
                          ("d3q19_foam_512", "f32", 16): 8 * 2534.55e6,
                          ("d3q19_foam_512", "f16", 24): 8 * 1264.90e6}
# FP64 storage: the step kernel is bound by the FP64 pipe, not by HBM.  FP64
# operations per lattice update of its D3Q19 kernel, DADD + DMUL + 2 DFMA as
# ncu counts them on the 128^3 case (146 + 71 + 2 x 332).  The peak is
# measured in the run by lbm_fp64_rate (a DFMA-chain kernel timed with CUDA
# events); the unit counts give 2 DFMA per SM and cycle x 152 SMs x 2 FLOP x
# 2.07 GHz = 1.26 TFLOP/s, used only if that measurement fails.
FP64_FLOP_PER_UPDATE = 881
FP64_PEAK_DERIVED_TFLOPS = 2 * 152 * 2 * 2.07e9 / 1e12
STORAGE_NAME = {"f32": "FP32", "f64": "FP64", "f16": "FP16-offset", "bf16": "BF16-offset"}
# D3Q19 tile ids of the x-pair kernel (fused_step_kernel_x2)
X_PAIR_TILES = range(14, 26)


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for k in ("hbm_gbs", "hbm_GBs", "hbm_bw_gbs", "hbm"):
            if k in d:
                v = d[k]
                if isinstance(v, dict):
                    v = v.get("burst", v.get("value"))
                return float(v), "measured"
        for k, v in d.items():
            if "hbm" in k.lower() and isinstance(v, (int, float)):
                return float(v), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    """One process per GPU (torch.distributed.run sets RANK, WORLD_SIZE,
    LOCAL_RANK, MASTER_*): NCCL on GPUs, gloo where there is none (the
    host-side logic of the N > 1 path is tested that way on CPU)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x):
    """The slowest rank's time: every rank gets the maximum."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, x):
    """The sum of x over the ranks: every rank gets it."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_lists(world, items):
    """The concatenation of every rank's list, on every rank."""
    if world == 1:
        return list(items)
    import torch.distributed as dist
    out = [None] * world
    dist.all_gather_object(out, list(items))
    return [x for part in out for x in part]


def ensemble_shard(domains, world, rank):
    """The domains of one rank: sorted by cells (largest first, ties by
    index) and dealt round-robin, so that every rank gets a like share of
    the cells; the ranks' shards are disjoint and cover all domains."""
    order = sorted(range(len(domains)), key=lambda d: (-domains[d]["nx"] * domains[d]["ny"], d))
    return [domains[d] for d in order[rank::world]]


def job_value(units_per_rank, world, seconds):
    """Whole-job throughput in millions of units per second: every rank
    processes units_per_rank (independent replicas), the job takes the
    slowest rank's seconds."""
    return units_per_rank * world / seconds / 1e6


FILM_H_MAX, FILM_EPS_ARM, FILM_CAP, CENSUS_BINS = 12, 1e-3, 4096, 32


def site_budgets(n):
    """Blowing-agent budget per site: a number, or (lo, hi) drawn uniformly
    from the recipe's seed."""
    b = W["budget"]
    if isinstance(b, tuple):
        return np.random.default_rng(W["seed"]).uniform(b[0], b[1], n)
    return np.full(n, float(b))


def resid():
    """The per-cell rounding residual of 16-bit storage, when the workload
    asks for it (FP32 and FP64 storage have none)."""
    return bool(W.get("mass_residual")) and W["storage"] in ("f16", "bf16")


def make_lattice(lbm, kernel="auto", tile=0):
    s = W["sites"]
    bub = lbm.sample_sites(W["nx"], W["ny"], W["nz"], s["n"], s["r_min"], s["r_max"],
                           s["min_spacing"], s["min_gap"], W["seed"])
    L = lbm.Lattice("D3Q19", W["nx"], W["ny"], W["nz"], tau=W["tau"], G=W["G"],
                    rho0=W["rho0"], storage=W["storage"], gas_threshold=W["threshold"],
                    rho_ref=W["rho_ref"], kernel="fused" if tile else kernel, tile=tile,
                    mass_residual=resid())
    L.seed_bubbles(bub, W["rho_l"], W["rho_g"], W["width"], W["noise"], W["seed"])
    rate = np.full(len(bub), W["rate"])
    budget = site_budgets(len(bub))
    L.inject(rate, budget)
    return L, rate, budget


def diagnostics(L):
    """The diagnostic interval through the C ABI (labels computed once);
    returns the number of gas components."""
    # FP64 totals + gas labels in one pass, site labels and merge events, the
    # film test at every lattice point, the bubble census: one call, one sync
    return L.diagnostic_interval(FILM_H_MAX, FILM_EPS_ARM, FILM_CAP, CENSUS_BINS)["ncomp"]


# kernels of one diagnostic interval (FP32 storage): scan + final (totals and
# gas flags), union + compress (labels), site gather, film test (one walk per
# lattice line and axis, then the queued midpoints with their pressure),
# census count + list
DIAG_LAUNCHES = 11


# The oracle's FP64 populations of a 512^3 or 768^3 lattice (20 GB, 68 GB)
# do not fit a bounded CPU sample, so the CPU legs step a 128^3 periodic
# lattice seeded by the same recipe, its bubble count scaled to the volume.
CPU_SAMPLE_SIDE = 128


def cpu_sample():
    """(side, bubbles, site cells, rates, budgets, description) of the
    lattice the oracle steps for the CPU legs: the workload itself up to
    128^3, else a 128^3 lattice with the same recipe (parameters, radius
    law, spacing rule, seed) and the bubble count scaled by volume."""
    import oracle as O
    s = W["sites"]
    side = min(W["nx"], CPU_SAMPLE_SIDE)
    n = s["n"] if side == W["nx"] else max(1, round(s["n"] * (side / W["nx"]) ** 3))
    got, bub = O.sample_sites(side, side, side, n, s["r_min"], s["r_max"], s["min_spacing"],
                              s["min_gap"], W["seed"])
    cells = (np.floor(bub[:, 0] + 0.5) + side * (np.floor(bub[:, 1] + 0.5)
             + side * np.floor(bub[:, 2] + 0.5))).astype(np.int64)
    rate = np.full(len(bub), W["rate"])
    budget = site_budgets(len(bub))
    what = ("the full %d^3 lattice" % side if side == W["nx"] else
            "a %d^3 periodic lattice of the %d^3 recipe (%d bubbles, the %d scaled by volume)"
            % (side, W["nx"], n, s["n"]))
    if W["rate"] > 0:
        what += " with injection"
    return side, bub, cells, rate, budget, what


def cpu_baseline(seconds_target=15.0):
    """The FP64 oracle on the host cores, bounded sample of the workload."""
    import oracle as O
    side, bub, cells, rate, budget, what = cpu_sample()
    f, _ = O.init(O.D3Q19, side, side, side, bub, W["rho_l"], W["rho_g"], W["width"],
                  W["noise"], W["seed"])
    O.run(O.D3Q19, f, 1, W["tau"], W["G"], sites=cells, rate=rate, budget=budget)  # warm
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds_target:
        f = O.run(O.D3Q19, f, 1, W["tau"], W["G"], sites=cells, rate=rate, budget=budget)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": side ** 3 * n / dt / 1e6, "unit": UNIT, "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{n} oracle time steps of {what} ({dt:.1f} s, OpenMP over all host "
                      f"cores)"}


def base_config():
    """The workload's config, the same for both arms."""
    return {"workload": W["name"], "lattice": "D3Q19", "extent": [W["nx"], W["ny"], W["nz"]],
            "storage": W["storage"], "mass_residual": resid(), "tau": W["tau"], "G": W["G"],
            "sites": W["sites"]["n"],
            "lbm_steps_per_bench_step": INNER, "rho_ref": W["rho_ref"],
            "l2": "inputs larger than L2: two %.0f MB population lattices"
                  % (CELLS * B_ALG / 2 / 1e6),
            "diagnostics": {"film_h_max": FILM_H_MAX, "film_eps_arm": FILM_EPS_ARM,
                            "census_bins": CENSUS_BINS}}


def run_reference(args, world, rank):
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    import oracle as O
    side, bub, cells, rate, budget, what = cpu_sample()
    f, _ = O.init(O.D3Q19, side, side, side, bub, W["rho_l"], W["rho_g"], W["width"],
                  W["noise"], W["seed"])
    for _ in range(warm):
        f = O.run(O.D3Q19, f, 1, W["tau"], W["G"], sites=cells, rate=rate, budget=budget)
    t0 = time.perf_counter()
    for _ in range(steps):
        f = O.run(O.D3Q19, f, 1, W["tau"], W["G"], sites=cells, rate=rate, budget=budget)
    dt = time.perf_counter() - t0
    val = side ** 3 * steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(base_config(),
                           sample=f"the FP64 oracle, one LBM time step of {what} per bench "
                                  f"step"),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{steps} oracle time steps of {what}"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    from paper_1708_01608_gb300 import build_lib
    if rank == 0 or not build_lib.up_to_date():
        build_lib.build()
    barrier(world)
    from paper_1708_01608_gb300 import lbm

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    L, rate, budget = make_lattice(lbm, args.kernel, args.tile)
    tuned = None
    if args.kernel != "two_pass" and not args.tile:
        tuned = L.autotune(10)  # set-up, outside the timed region; state is restored
    plan = L.plan()

    gas = []  # gas components found by each timed interval

    def bench_step(e_begin=None, e_end=None):
        if e_begin is not None:
            e_begin.record(stream)
        L.step(INNER)
        if e_end is not None:
            e_end.record(stream)
        return diagnostics(L)

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()

    # ---- device-resident timed region
    clocks = ClockSampler(local)
    clocks.start()
    ev_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    t_start.record(stream)
    for k in range(args.steps):
        gas.append(bench_step(*ev_step[k]))
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = t_start.elapsed_time(t_end)
    ms = max_over_ranks(world, ms)
    step_kernel_ms = sum(a.elapsed_time(b) for a, b in ev_step) / (args.steps * INNER)

    # ---- end to end through the C ABI with host buffers (pinned)
    labels = torch.empty(L.shape, dtype=torch.int32, pin_memory=True).numpy()
    rate_h = torch.tensor(rate, dtype=torch.float64).pin_memory().numpy()
    budget_h = L.read_budgets()
    budget_pin = torch.tensor(budget_h, dtype=torch.float64).pin_memory().numpy()
    rec = torch.empty(FILM_CAP * lbm.FILM_CELL.itemsize, dtype=torch.uint8,
                      pin_memory=True).numpy()
    roots = torch.empty(1 << 16, dtype=torch.int64, pin_memory=True).numpy()
    sizes = torch.empty(1 << 16, dtype=torch.int64, pin_memory=True).numpy()
    hist = np.zeros(CENSUS_BINS, dtype=np.int64)
    import ctypes as C
    rep = lbm.IntervalReport()
    vp = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        L.inject(rate_h, budget_pin)                      # H2D: rates and budgets
        L.step(INNER)
        # D2H: totals, labels, film census and fired cells, bubble census
        lbm._check(lbm.lib().lbm_diagnostic_interval(
            L.handle, FILM_H_MAX, FILM_EPS_ARM, vp(labels), vp(rec), FILM_CAP, vp(roots),
            vp(sizes), len(roots), vp(hist), CENSUS_BINS, C.byref(rep)))
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    h2d = rate_h.nbytes + budget_pin.nbytes
    # the results handed out per step: labels, totals, component count, film
    # counts and fired cells, census entries and histogram
    d2h = (labels.nbytes + 32 + 8 + 32 + lbm.FILM_CELL.itemsize * int(rep.nfired)
           + 16 * int(rep.nsizes) + hist.nbytes)

    units = CELLS * INNER * args.steps  # per rank
    value = job_value(units, world, ms / 1e3)
    e2e_val = job_value(units, world, e2e_s)
    peak, src = peak_hbm()
    achieved = B_ALG * CELLS / (step_kernel_ms / 1e3) / 1e9
    traffic = NCU_TRAFFIC_PER_LAUNCH.get((W["name"], W["storage"] + ("+resid" if resid() else ""),
                                          plan[1]))
    kname = "fused_step_kernel_x2" if plan[1] in X_PAIR_TILES else "fused_step_kernel"
    if W["storage"] == "f64":
        tflops = FP64_FLOP_PER_UPDATE * CELLS / (step_kernel_ms / 1e3) / 1e12
        try:
            fp64_peak = lbm.fp64_rate()
            fp64_src = ("measured in this run: DFMA-chain kernel over every SM "
                        "(lbm_fp64_rate, CUDA events, fastest of 3)")
        except lbm.LBMError:
            fp64_peak = FP64_PEAK_DERIVED_TFLOPS
            fp64_src = "derived from unit counts and the 2.07 GHz clock"
        roofline = {"bound": "alu", "achieved": tflops, "peak": fp64_peak,
                    "unit": "TFLOP/s", "frac": tflops / fp64_peak,
                    "peak_source": fp64_src,
                    "traffic": traffic, "kernel": kname, "flop_per_update": FP64_FLOP_PER_UPDATE,
                    "bytes_per_update": B_ALG, "kernel_ms": step_kernel_ms}
    else:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_source": src, "traffic": traffic,
                    "kernel": kname, "bytes_per_update": B_ALG, "kernel_ms": step_kernel_ms}
    launches_per_step = INNER + DIAG_LAUNCHES
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if W["storage"] == "f64" else "f32",
            "data": "synthetic",
            "config": dict(base_config(), kernel=args.kernel,
                           plan={"kernel": plan[0], "tile": plan[1], "tile_xy": [plan[2], plan[3]],
                                 "z_chunks": plan[4], "ctas": plan[5]},
                           parallelism=f"replicas x{world}",
                           rho_l=W["rho_l"],
                           gas_components={"per_timed_interval": gas,
                                           "min": min(gas) if gas else None},
                           lbm_steps_before_timing=INNER * args.warmup),
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    L.close()


def run_ensemble(args, world=1, rank=0, local=0):
    """The batched two-bubble sweep (256 uneven D2Q9 domains) run until every
    criterion fired or 20000 steps; MLUPS over all domain updates.  With N
    ranks the domains are sharded over the GPUs (independent problems, no
    exchange): the job's time is the slowest rank's, its updates the sum."""
    import torch
    from paper_1708_01608_gb300 import build_lib
    from paper_1708_01608_gb300 import workloads as WL
    if rank == 0 or not build_lib.up_to_date():
        build_lib.build()
    barrier(world)
    from paper_1708_01608_gb300 import lbm
    torch.cuda.set_device(local)
    R = WL.ENSEMBLE_256
    all_doms = WL.ensemble_domains(R)
    doms = ensemble_shard(all_doms, world, rank)
    def sweep():
        # one bench step: a fresh ensemble of the same domains run to completion;
        # set-up is outside the timed region, the sweep inside it
        E = lbm.Ensemble(doms, eps_arm=R["eps_arm"], diag_every=R["diag_every"],
                         h_max=R["h_max"])
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E.run(R["steps"])
        torch.cuda.synchronize()
        return E, max_over_ranks(world, time.perf_counter() - t0)

    for _ in range(args.warmup):
        sweep()[0].close()
    clocks = ClockSampler(local)
    clocks.start()
    dt, upd = 0.0, 0.0
    for k in range(args.steps):
        E, t = sweep()
        dt += t
        upd += E.stats()["updates"]
        if k + 1 < args.steps:
            E.close()
    clk = clocks.stop()
    barrier(world)
    st = E.stats()
    res = E.results()
    updates = sum_over_ranks(world, upd)
    fired = gather_lists(world, [(d["R"], r["h_c"], r["r_d"], r["steps"])
                                 for d, r in zip(doms, res) if r["fired"]])
    fired.sort()
    merged = int(sum_over_ranks(world, sum(r["merged"] for r in res)))
    launches = int(sum_over_ranks(world, st["launches"]))
    steps = int(max_over_ranks(world, st["steps"]))
    line = {"metric": "batched D2Q9 ensemble MLUPS (256 two-bubble domains, run to the rupture "
                      "criterion or 20000 steps)",
            "value": updates / dt / 1e6, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / max(args.steps, 1) * 1e3,
            "higher_is_better": True, "scaling": "strong", "dtype": "f32", "data": "synthetic",
            "config": {"workload": R["name"], "domains": len(all_doms),
                       "cells": int(sum(d["nx"] * d["ny"] for d in all_doms)),
                       "lbm_steps_per_sweep": steps, "bench_step": "one sweep run to completion",
                       "diag_every": R["diag_every"], "eps_arm": R["eps_arm"], "h_max": R["h_max"],
                       "l2": "inputs larger than L2: 1.16 GB of populations",
                       "parallelism": f"domains sharded over {world} GPU(s)"},
            "seconds": dt, "updates": updates, "launches_per_sweep": launches,
            "gpu_launches": launches * args.steps, "clocks": clk,
            "fired": len(fired), "merged": merged,
            "h_c_vs_R": [[round(a, 2), round(b, 3), round(c, 1), s] for a, b, c, s in fired]}
    if len(fired) >= 3:
        # the functional forms of Fig. 3 fitted to the fired domains (R_b = disk radius)
        from paper_1708_01608_gb300.sweep import fit_fig3
        line["fig3_fit"] = fit_fig3([a for a, _, _, _ in fired], [c for _, _, c, _ in fired],
                                    [b for _, b, _, _ in fired])
    E.close()
    if rank != 0:
        return
    if args.single and world == 1:
        upd, t_single = 0.0, 0.0
        for dm in doms:
            L = lbm.Lattice("D2Q9", dm["nx"], dm["ny"], 1, tau=dm["tau"], G=dm["G"],
                            storage="f32", rho_ref=dm["rho_ref"], kernel="fused")
            L.seed_bubbles(np.array(dm["bubbles"]), dm["rho_l"], dm["rho_g"], dm["width"],
                           dm["noise_amp"], dm["seed"])
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            r = L.run_until_rupture(dm["line"], dm["rho_mid"], R["eps_arm"], R["diag_every"],
                                    R["steps"], R["h_max"])
            t_single += time.perf_counter() - t1
            upd += dm["nx"] * dm["ny"] * r["steps"]
            L.close()
        line["single_domain_mlups"] = upd / t_single / 1e6
        line["single_domain_seconds"] = t_single
    print(json.dumps(line), flush=True)


def run_ml_sweep(args, world=1, rank=0, local=0):
    """Nine bubble sizes (Sec. 4, Fig. 3) in the multi-lattice model and in
    the single-component model: per size, the two disks run until the
    rupture criterion fires (eta_m = 0 merges the pair's lattices) or the
    film is gone; h_c against R_d beside the paper's fitted forms.  Not a
    throughput line: every domain runs once, and the rank-0 process alone
    does the work."""
    import torch
    from paper_1708_01608_gb300 import build_lib
    from paper_1708_01608_gb300 import workloads as WL
    if rank != 0:
        return
    build_lib.build()
    from paper_1708_01608_gb300 import lbm
    torch.cuda.set_device(local)
    R = WL.ML_SWEEP_9
    rows = {"multi_lattice": [], "single_component": []}
    t0 = time.perf_counter()
    updates = 0.0
    for dm in WL.ml_sweep_domains(R):
        L = dm["L"]
        b = np.array(dm["bubbles"])
        mid = 0.5 * (R["rho_l"] + R["rho_v"])
        M = lbm.MultiLattice("D2Q9", L, L, 1, nl=3, tau=R["tau"], rho0=R["rho0"], G=R["G"],
                             G_x=R["G_x"], G_b=R["G_b"], storage="f64")
        M.seed(b, R["rho_l"], R["rho_v"], R["rho_gas"], R["width"], R["noise"], R["seed"])
        r = M.run_until_rupture(dm["line"], mid, R["eps_arm"], R["diag_every"], R["steps"],
                                R["h_max"])
        rows["multi_lattice"].append(dict(R_b=dm["R"], L=L, **r))
        updates += 3.0 * L * L * r["steps"]
        M.close()
        S = lbm.Lattice("D2Q9", L, L, 1, tau=R["tau"], G=R["G"], rho0=R["rho0"], storage="f64",
                        kernel="fused")
        S.seed_bubbles(b, R["rho_l"], R["rho_v"], R["width"], R["noise"], R["seed"])
        r = S.run_until_rupture(dm["line"], mid, R["eps_arm"], R["diag_every"], R["steps"],
                                R["h_max"])
        rows["single_component"].append(dict(R_b=dm["R"], L=L, **r))
        updates += L * L * r["steps"]
        S.close()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    from paper_1708_01608_gb300.sweep import fit_fig3
    fits = {}
    for k, rr in rows.items():
        fired = [x for x in rr if x["fired"]]
        if len(fired) >= 3:
            fits[k] = fit_fig3([x["R_b"] for x in fired], [x["r_d"] for x in fired],
                               [x["h_c"] for x in fired])
    line = {"metric": "nine-size two-bubble sweep, multi-lattice vs single-component Shan-Chen "
                      "(h_c vs R_d; not a throughput line)",
            "value": updates / dt / 1e6, "unit": "MLUPS (lattice updates incl. every lattice)",
            "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "seconds": dt,
            "config": {"workload": R["name"], "radii": list(R["radii"]), "gap": R["gap"],
                       "tau": R["tau"], "G": R["G"], "G_x": R["G_x"], "G_b": R["G_b"],
                       "rho_gas": R["rho_gas"], "noise": R["noise"],
                       "diag_every": R["diag_every"], "eps_arm": R["eps_arm"],
                       "h_max": R["h_max"], "max_steps": R["steps"]},
            "rows": {k: [{q: (round(v, 4) if isinstance(v, float) else v) for q, v in x.items()}
                         for x in rr] for k, rr in rows.items()},
            "fig3_fit": fits,
            "paper_fit": {"h_c": "0.002 R_d^2 - 0.003 R_d + 0.035",
                          "R_d": "2.088 ln(R_b) + 0.114", "units": "the paper's (unstated)"}}
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    import torch
    from paper_1708_01608_gb300 import build_lib
    build_lib.build()
    from paper_1708_01608_gb300 import lbm
    torch.cuda.set_device(0)
    s = W["sites"]
    n = args.extent or W["nx"]
    storage = args.storage or W["storage"]
    bub = lbm.sample_sites(n, n, n, s["n"], s["r_min"], s["r_max"], s["min_spacing"],
                           s["min_gap"], W["seed"])
    L = lbm.Lattice("D3Q19", n, n, n, tau=W["tau"], G=W["G"], rho0=W["rho0"], storage=storage,
                    rho_ref=W["rho_ref"], kernel="fused" if args.tile else args.kernel,
                    tile=args.tile)
    L.seed_bubbles(bub, W["rho_l"], W["rho_g"], W["width"], W["noise"], W["seed"])
    L.inject(np.full(len(bub), W["rate"]), site_budgets(len(bub)))
    L.step(args.profile_steps)
    if args.profile_diagnostics:
        diagnostics(L)  # one diagnostic interval after the steps
    L.sync()
    print(json.dumps({"profile_case": W["name"], "extent": n, "storage": storage,
                      "steps": args.profile_steps, "diagnostics": args.profile_diagnostics,
                      "plan": L.plan()}))
    L.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "fused", "two_pass"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="no timing: build the workload lattice, run this many steps, exit "
                         "(a short fixed case for ncu captures)")
    ap.add_argument("--tile", type=int, default=0,
                    help="fused tile id: for --profile-steps, or for a timed run without the "
                         "autotuner (a launch-list capture under ncu, whose serialised "
                         "launches would mislead the autotuner's timing)")
    ap.add_argument("--extent", type=int, default=0,
                    help="--profile-steps: cubic lattice side (default: the workload's)")
    ap.add_argument("--profile-diagnostics", action="store_true",
                    help="--profile-steps: then run one diagnostic interval")
    ap.add_argument("--workload", default=None,
                    choices=["foam128", "foam512", "foam768", "ensemble256", "ml9"],
                    help="foam512: the default benchmark line, the 512^3 foam (FP32, or "
                         "--storage f16/bf16/f64); foam128: 64 injecting nuclei on 128^3 (the "
                         "default of --profile-steps, whose --extent keeps its 64 sites); "
                         "foam768: the 768^3 FP16-offset full foam with 4096 injection sites; "
                         "ensemble256: the batched two-bubble sweep run to completion; ml9: "
                         "nine bubble sizes in the multi-lattice and the single-component "
                         "model (h_c vs R_d, not a throughput line)")
    ap.add_argument("--storage", default=None, choices=["f32", "f16", "bf16", "f64"])
    ap.add_argument("--single", action="store_true",
                    help="ensemble256: also run every domain alone, one after the other")
    args = ap.parse_args()
    global W, METRIC, CELLS, B_ALG
    from paper_1708_01608_gb300 import workloads as WL
    if args.workload is None:
        args.workload = "foam128" if args.profile_steps > 0 else "foam512"
    if args.workload == "foam128":
        W = dict(WL.FOAM_128)
        METRIC = ("D3Q19 Shan-Chen MLUPS (128^3 foam, FP32 storage, 64 sites, injection + "
                  "diagnostics every 100 steps)")
    elif args.workload == "foam768":
        W = dict(WL.FOAM_768)
        METRIC = ("D3Q19 Shan-Chen MLUPS (768^3 full foam, FP16-offset storage, 4096 sites "
                  "with injection, diagnostics every 100 steps)")
    CELLS = W["nx"] * W["ny"] * W["nz"]
    if args.profile_steps > 0:
        run_profile_case(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup(args.gpus)
    if args.workload == "ml9":
        try:
            run_ml_sweep(args, world, rank, local)
        finally:
            if world > 1:
                import torch.distributed as dist
                dist.destroy_process_group()
        return
    if args.workload == "ensemble256":
        try:
            run_ensemble(args, world, rank, local)
        finally:
            if world > 1:
                import torch.distributed as dist
                dist.destroy_process_group()
        return
    if args.storage:
        # the metric names the storage form measured
        METRIC = METRIC.replace(STORAGE_NAME[W["storage"]], STORAGE_NAME[args.storage])
        W = dict(W, storage=args.storage)
    # bytes per lattice update: every population read and written once, plus
    # the rounding residual's FP32 read and write when 16-bit storage keeps one
    B_ALG = 2 * Q * {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[W["storage"]] + (8 if resid() else 0)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
