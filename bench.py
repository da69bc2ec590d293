#!/usr/bin/env python
"""Throughput of the tCW template-bank track-statistic search on GB300.

One step = one full search (Doppler table, track entries + gather + weighted
sum + Psi, per-sky top-100) of the plain 2-detector workload: 10^4 segments x
10^4 bins fp32 power (T_SFT = 4 s, 500-3000 Hz) with 10 injected tracks, a
uniform-random bank of 2e5 (f0, tau, n) templates and 1024 Fibonacci-sphere sky
directions.  Unit of work: one template.segment sum = one (template, sky,
detector, segment) lookup; a step is 2e5 * 1024 * 2 * 10^4 = 4.1e12 of them.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank searches its own 1024-sky slice of an N*1024-point
sky lattice over the same data (weak scaling, no data-path collective); the
step time is the maximum over ranks.  Rank 0 prints one JSON line.

On one GPU the line also carries further forms of the search, each on its
own synthetic workload:
  "small"    the 1-detector 256 x 4096 map, 5120 lattice templates, 1 sky, with
             the FP64 oracle timed on the whole of it
  "batched"  64 events of 2000-20000 segments x 10^4 FP16 bins, own T0 and
             256-4096 skies each, against a 2e4-template bank, in one
             graph-replayed persistent launch (autotuned shapes)
  "learned"  the triaged search (coarse pass on every segment, network,
             best 35 % of the sky patches with their best 1.2 % of templates)
             against the exhaustive one on 100 held-out 2-detector 10^4 x 10^4
             events with one injection each and the full 2e5-template bank,
             judged by the exhaustive search with the noise-only maximum of Psi
             as the detection threshold (Sec. 3)
  "batched_learned"  the batched triaged search (one coarse pass per event,
             one network call, one launch over the chosen items) against the
             exhaustive batched search of the same 16 events (2000-20000
             segments x 10^4 bins, 2 detectors, 1024 skies, 2e5 templates, one
             injection each), judged by the exhaustive batched search
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "template·segment sums/s"
UNIT = "sums/s"
TOPK = 100


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="full", choices=["full", "small", "scaled", "bank8000"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-amplitude", action="store_true",
                    help="skip the generated-bank, amplitude, count and two-bin variants")
    ap.add_argument("--batched-events", type=int, default=64)
    ap.add_argument("--batched-templates", type=int, default=20000)
    ap.add_argument("--learned-events", type=int, default=100)
    ap.add_argument("--batched-learned-events", type=int, default=16)
    return ap.parse_args()


def rank_sky(rank, world, per_rank=1024):
    """Rank `rank`'s slice of an equal-area lattice of world * per_rank skies
    (weak scaling: every rank searches its own skies over the same data)."""
    import tcw_synth as syn
    return np.ascontiguousarray(syn.fibonacci_sky(per_rank * world)[rank * per_rank:(rank + 1) * per_rank])


def max_over_ranks(x, dist=None, device=None):
    """The largest x over the ranks (the job's time is its slowest rank's)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, steps, seconds):
    """Whole-job throughput: the units every rank processed / the max-over-ranks time."""
    return world * units_per_rank * steps / seconds


def make_problem(workload, rank, world):
    import tcw_synth as syn
    if workload == "small":
        p = syn.config_small(seed=20250711, weights=True)
        return p
    if workload == "scaled":
        # the full workload cut to 2000 segments and 8000 templates (profiling case)
        return syn.config_full(seed=20250712, n_seg=2000, n_tmpl=8000, n_inj=2)
    if workload == "bank8000":
        # the full workload with the bank cut to 8000 templates: every segment, so
        # the Doppler table (100 MB) and the map (800 MB) are the full ones
        # (DRAM-traffic case: one launch is 1/25 of a full one)
        return syn.config_full(seed=20250712, n_tmpl=8000)
    p = syn.config_full(seed=20250712)
    if world > 1:
        p.nhat = rank_sky(rank, world)
    return p


def units(p):
    D, Nseg, _ = p.rho.shape
    return int(p.nhat.shape[0]) * len(p.bank) * D * Nseg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_uuid=None):
        self.proc = None
        self.uuid = dev_uuid

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["--id=" + self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_digest():
    """First 16 hex digits of the sha256 of the group kernel's sources
    (tcw_persist.cuh followed by tcw_ptx.cuh)."""
    h = hashlib.sha256()
    for f in ("tcw_persist.cuh", "tcw_ptx.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2507_07816_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


# DRAM bytes (read + write) of one group-kernel launch per lookup, from an ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum, one pass) of the
# bank8000 workload: the full 2 x 10000 x 10000 map, Doppler table and sky with
# 8000 templates, one launch; a full launch streams the same map and table once
# per pass, 25 times as many passes, so it is taken to move the same bytes per
# lookup.  Keyed by the kernel source digest it was taken on; no entry for the
# current source: the traffic is reported as null.
GROUP_KERNEL_DRAM_BYTES_PER_LOOKUP = {
    "c816dee2c7d44e5e": (3010211584 + 39771392) / (1024 * 8000 * 2 * 10000),
}


def group_kernel_traffic(lookups):
    per = GROUP_KERNEL_DRAM_BYTES_PER_LOOKUP.get(kernel_source_digest())
    return None if per is None else per * lookups


def oracle_rate(p, seconds, seed=0):
    """Oracle lookups/s on a bounded sample of (sky, template) pairs of p."""
    import oracle
    D, Nseg, _ = p.rho.shape
    r = np.random.default_rng(seed)
    S, B = p.nhat.shape[0], len(p.bank)

    def run(npairs):
        pairs = np.stack([r.integers(0, S, npairs), r.integers(0, B, npairs)], 1)
        t0 = time.perf_counter()
        oracle.search_stats(p.rho, p.f_min, p.df, p.t_mid, p.weights, p.velocity, p.nhat,
                            p.bank.f0, p.bank.tau, p.bank.n, p.T0, pairs=pairs)
        return time.perf_counter() - t0

    threads = oracle.max_threads()
    n = max(threads * 2, 16)
    dt = run(n)
    while dt < 1.0 and n < 2_000_000:          # calibrate on about a second of work
        n = min(2_000_000, n * 4)
        dt = run(n)
    n = int(min(max(n, n * seconds / max(dt, 1e-6)), 2_000_000))
    dt = run(n)
    lookups = n * D * Nseg
    return lookups / dt, threads, n, dt


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def bench_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p = make_problem(args.workload, 0, 1)
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    rates = []
    for i in range(args.warmup + args.steps):
        rate, threads, n, dt = oracle_rate(p, per_step, seed=i)
        if i >= args.warmup:
            rates.append(rate)
    D, Nseg, _ = p.rho.shape
    value = float(statistics.mean(rates))
    sample = (f"{n} random (sky, template) pairs x {D} detectors x {Nseg} segments per step "
              f"of the {p.name} workload")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * units(p) / value,
        "extrapolated": True,
        "ms_per_step_basis": (f"time of one whole step at the rate measured on {n} sampled (sky, template) "
                              f"pairs per step ({n * D * Nseg:.3g} of the step's {units(p):.3g} sums)"),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": p.name, "implementation": "FP64 C oracle (OpenMP)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample, "cpu": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def bench_batched(args, dev):
    """Batched search of the 64-event workload: device time of a graph replay."""
    import torch
    import paper_2507_07816_gb300 as tcw
    import tcw_synth as syn
    t0 = time.perf_counter()
    events, bank = syn.config_batched(n_events=args.batched_events, n_tmpl=args.batched_templates,
                                      device=torch.device(f"cuda:{dev}"))
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    s = tcw.Search(dev)
    s.define_bank(bank.f0, bank.tau, bank.n, 0.0)
    s.load_events(events, events[0].f_min, events[0].df)
    t0 = time.perf_counter()
    s.search_batched(TOPK)           # plans, autotunes and records the graph
    first_s = time.perf_counter() - t0
    ms, walls = [], []
    for _ in range(2):
        t0 = time.perf_counter()
        val, idx = s.search_batched(TOPK)
        walls.append(time.perf_counter() - t0)
        ms.append(s.batch_info()["search_ms"])
    info = s.batch_info()
    row, hit = 0, 0
    for e in events:
        inj = e.injections[0]
        srow = int(np.nonzero(np.all(e.nhat == inj.nhat, axis=1))[0][0])
        hit += int(inj.template in idx[row + srow, :10].tolist())
        row += e.nhat.shape[0]
    s.close()
    # the same events searched one by one by the plain search (wall time of a
    # second search of each event: Doppler, anchors, group kernel, top-k, copy out)
    plain_wall = 0.0
    s1 = tcw.Search(dev)
    for e in events:
        s1.load_problem(e)
        s1.search(TOPK)
        t0 = time.perf_counter()
        s1.search(TOPK)
        plain_wall += time.perf_counter() - t0
    s1.close()
    n_seg = [int(e.rho.shape[1]) for e in events]
    skies = [int(e.nhat.shape[0]) for e in events]
    dev_ms = statistics.mean(ms)
    out = {"workload": f"batched-{len(events)}ev-{min(n_seg)}..{max(n_seg)}seg-x10000-f16-"
                       f"sky{min(skies)}..{max(skies)}-bank{len(bank)}",
           "value": info["lookups"] / (dev_ms / 1000.0), "unit": UNIT, "search_ms": dev_ms,
           "wall_ms": 1000.0 * statistics.mean(walls), "lookups": info["lookups"],
           "first_call_s": first_s, "generate_s": gen_s, "events": len(events),
           "injections_top10": f"{hit}/{len(events)}",
           "plain_same_events": {"value": info["lookups"] / plain_wall, "unit": UNIT, "wall_ms": 1000.0 * plain_wall,
                                 "basis": "tcw_search of each event in turn, wall time of its second search"},
           "vs_plain_same_events": plain_wall / statistics.mean(walls)}
    for key in ("waves", "bank_chunk", "tile_segments", "autotuned", "n_candidates", "n_items",
                "graph_kernels", "tune_ms", "best_rate", "default_rate"):
        out[key] = info[key]
    return out


def bench_learned(args, dev):
    """Triaged vs exhaustive search on held-out events, judged by the exhaustive one."""
    import torch
    import paper_2507_07816_gb300 as tcw
    from paper_2507_07816_gb300 import triage as TR
    import tcw_synth as syn
    wpath = os.path.join(ROOT, "paper_2507_07816_gb300", "triage_weights.npz")
    if not os.path.exists(wpath):
        return {"skipped": "no trained weights (paper_2507_07816_gb300/triage_weights.npz)"}
    meta = dict(np.load(wpath, allow_pickle=False))
    bank = syn.random_bank(syn.rng(int(meta["bank_seed"])), int(meta["n_tmpl"]), f0_range=(500.0, 3000.0))
    mlp = tcw.Mlp.load(wpath, device=f"cuda:{dev}")
    seed0 = int(meta["valid_seed"]) + 10_000

    def make(i):
        return syn.training_event(seed0 + i, bank, n_inj=int(meta["injections"]), snr_range=(6.0, 12.0),
                                  device=torch.device(f"cuda:{dev}"))

    stride = int(meta["stride"]) if "stride" in meta else 1
    psi_det = float(meta["psi_det"]) if "psi_det" in meta else 6.5
    # one untimed event first: buffers, library state and the subset bank path warm up
    TR.evaluate(mlp, lambda i: make(10**6 + i), 1, bank, psi_det, frac=TR.FRAC, patch_size=int(meta["patch_size"]),
                k=TOPK, templates_permille=TR.TEMPLATES_PERMILLE, stride=stride)
    r = TR.evaluate(mlp, make, args.learned_events, bank, psi_det, frac=TR.FRAC,
                    patch_size=int(meta["patch_size"]), k=TOPK, templates_permille=TR.TEMPLATES_PERMILLE,
                    stride=stride)
    r["value"] = r["sums_full"] / r["time_triaged_s"]
    r["unit"] = UNIT
    r["plain_value"] = r["sums_full"] / r["time_full_s"]
    r["workload"] = f"learned-2det-10000x10000-bank{len(bank)}-sky1024"
    r["judge"] = ("exhaustive search of every sky; found = injected template in the first 10 of a sky within 64 "
                  "Doppler-sorted positions with Psi above the noise-only maximum psi_det (Sec. 3)")
    return r


def sorted_positions_of(ev):
    """Position of every sky of an event in the library's Doppler-sorted order
    (key: v.nhat of detector 0 at the middle segment, stable)."""
    vm = np.asarray(ev.velocity[0][ev.rho.shape[1] // 2], np.float64)
    order = np.argsort(np.asarray(ev.nhat, np.float64) @ vm, kind="stable")
    pos = np.empty_like(order)
    pos[order] = np.arange(order.shape[0])
    return pos


def bench_batched_learned(args, dev):
    """Batched triaged search against the exhaustive batched search of the same
    events (uneven segment counts, own start time and T0, one injection each),
    effective rate = the exhaustive search's sums / wall time of the triaged call,
    loss judged by the exhaustive batched search."""
    import torch
    import paper_2507_07816_gb300 as tcw
    from paper_2507_07816_gb300 import triage as TR
    import tcw_synth as syn
    wpath = os.path.join(ROOT, "paper_2507_07816_gb300", "triage_weights.npz")
    if not os.path.exists(wpath):
        return {"skipped": "no trained weights (paper_2507_07816_gb300/triage_weights.npz)"}
    meta = dict(np.load(wpath, allow_pickle=False))
    bank = syn.random_bank(syn.rng(int(meta["bank_seed"])), int(meta["n_tmpl"]), f0_range=(500.0, 3000.0))
    mlp = tcw.Mlp.load(wpath, device=f"cuda:{dev}")
    psi_det = float(meta["psi_det"]) if "psi_det" in meta else 6.5
    stride = int(meta["stride"]) if "stride" in meta else 1
    ps = int(meta["patch_size"])
    seed0 = int(meta["valid_seed"]) + 20_000
    n_segs = syn.rng(seed0).integers(2000, 20001, args.batched_learned_events)
    t0 = time.perf_counter()
    events = [syn.training_event(seed0 + i, bank, n_seg=int(n_segs[i]), n_inj=1, snr_range=(6.0, 12.0),
                                 device=torch.device(f"cuda:{dev}")) for i in range(len(n_segs))]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    s = tcw.Search(dev)
    s.set_option(tcw.OPT_TRIAGE_TEMPLATES, TR.TEMPLATES_PERMILLE)
    s.set_option(tcw.OPT_TRIAGE_STRIDE, stride)
    s.define_bank(bank.f0, bank.tau, bank.n, 0.0)
    s.load_events(events, events[0].f_min, events[0].df)
    t0 = time.perf_counter()
    s.search_batched(TOPK)              # plans, autotunes and records the graph
    first_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    vx, ix = s.search_batched(TOPK)
    wall_x = time.perf_counter() - t0
    sums_full = s.batch_info()["lookups"]
    s.search_batched_triaged(mlp, ps, TR.PSI_LO, TR.PSI_HI, TR.FRAC, TOPK)   # buffers warm up
    walls = []
    for _ in range(2):
        t0 = time.perf_counter()
        pt, it, searched = s.search_batched_triaged(mlp, ps, TR.PSI_LO, TR.PSI_HI, TR.FRAC, TOPK)
        walls.append(time.perf_counter() - t0)
    info = s.triage_info()
    s.close()
    found_x = found_t = missed = 0
    row = 0
    for e in events:
        S = e.nhat.shape[0]
        pos = sorted_positions_of(e)
        fx = TR.judge(e, vx[row:row + S], ix[row:row + S], pos, psi_det)
        ft = TR.judge(e, pt[row:row + S], it[row:row + S], pos, psi_det)
        found_x += sum(fx)
        found_t += sum(ft)
        missed += sum(a and not b for a, b in zip(fx, ft))
        row += S
    wall_t = min(walls)
    return {"workload": f"batched-learned-{len(events)}ev-{int(n_segs.min())}..{int(n_segs.max())}seg-"
                        f"2det-x10000-f32-sky1024-bank{len(bank)}",
            "value": sums_full / wall_t, "unit": UNIT, "plain_value": sums_full / wall_x,
            "speedup": wall_x / wall_t, "wall_triaged_s": wall_t, "wall_exhaustive_s": wall_x,
            "sums_full": sums_full,
            "sums_executed_triaged": info["lookups_coarse"] + info["lookups_searched"],
            "coarse_ms": info["coarse_ms"], "mlp_ms": info["mlp_ms"], "search_ms": info["search_ms"],
            "skies_searched": info["skies_searched"], "templates_searched": info["templates_searched"],
            "coarse_kernel": "sweep" if info["coarse_kernel"] else "per pair",
            "events": len(events), "detected_exhaustive": found_x, "detected_triaged": found_t,
            "missed": missed, "loss": missed / max(found_x, 1), "psi_det": psi_det,
            "frac": TR.FRAC, "templates_permille": TR.TEMPLATES_PERMILLE, "patch_size": ps, "stride": stride,
            "first_exhaustive_call_s": first_s, "generate_s": gen_s,
            "judge": ("the exhaustive batched search of every sky; found = injected template in the first 10 of "
                      "a sky within 64 Doppler-sorted positions with Psi above psi_det (Sec. 3)")}


def bench_small(args, dev):
    """The 1-detector 256 x 4096 workload (5120 lattice templates, 1 sky): device
    time of the search, and the FP64 oracle on the whole workload."""
    import torch
    import paper_2507_07816_gb300 as tcw
    import oracle
    p = make_problem("small", 0, 1)
    U = units(p)
    s = tcw.Search(dev)
    s.load_problem(p)
    for _ in range(3):
        s.search(TOPK)
    torch.cuda.synchronize()
    ms = []
    for _ in range(max(3, args.steps)):
        s.search(TOPK)
        ms.append(s.info().search_ms)
    kernel = {1: "group", 2: "lookup"}.get(s.info().kernel, "?")
    s.close()
    t0 = time.perf_counter()
    oracle.search_stats(p.rho, p.f_min, p.df, p.t_mid, p.weights, p.velocity, p.nhat, p.bank.f0, p.bank.tau,
                        p.bank.n, p.T0)
    dt = time.perf_counter() - t0
    dev_ms = statistics.median(ms)
    return {"workload": p.name, "value": U / (dev_ms / 1000.0), "unit": UNIT, "search_ms": dev_ms,
            "kernel": kernel, "lookups": U,
            "cpu_baseline": {"value": U / dt, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"the whole workload ({U} sums, {dt:.3f} s)"}}


def bench_ours(args):
    import torch
    import paper_2507_07816_gb300 as tcw

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group(backend="nccl")
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)

    p = make_problem(args.workload, rank, world)
    U = units(p)
    stream = torch.cuda.Stream(device=dev)
    s = tcw.Search(dev, stream=stream)
    s.load_problem(p)
    S = p.nhat.shape[0]
    k = min(TOPK, len(p.bank))
    psi_out = torch.empty((S, k), dtype=torch.float32, device=f"cuda:{dev}")
    idx_out = torch.empty((S, k), dtype=torch.int64, device=f"cuda:{dev}")

    def barrier():
        if dist:
            dist.barrier()

    for _ in range(args.warmup):
        s.search(k, psi_out, idx_out)
    torch.cuda.synchronize()
    barrier()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clk = ClockSampler(uuid)
    clk.start()
    time.sleep(0.5)
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    kernel_ms, launches = [], 0
    e0.record(stream)
    for _ in range(args.steps):
        s.search(k, psi_out, idx_out)
        inf = s.info()
        kernel_ms.append(inf.search_ms)
        launches += inf.launches
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    elapsed = max_over_ranks(e0.elapsed_time(e1), dist, f"cuda:{dev}")
    ms_per_step = elapsed / args.steps
    value = job_rate(world, U, args.steps, elapsed / 1000.0)
    info = s.info()

    # end to end through the public API: host (pinned) inputs in, host top-k out
    e2e = None
    if not args.no_e2e:
        rho_h = torch.from_numpy(p.rho).pin_memory()
        v_h = torch.from_numpy(np.ascontiguousarray(p.velocity)).pin_memory()
        w_h = None if p.weights is None else np.ascontiguousarray(p.weights)
        h2d = (rho_h.numel() * rho_h.element_size() + p.t_mid.nbytes
               + (0 if w_h is None else w_h.nbytes) + v_h.numel() * 8 + 3 * len(p.bank) * 8 + S * 3 * 8)
        d2h = S * k * (4 + 8)
        s2 = tcw.Search(dev, stream=stream)

        def e2e_step():
            s2.load_spectrogram(rho_h, p.f_min, p.df, p.t_mid, w_h)
            s2.load_velocity(v_h)
            s2.define_bank(p.bank.f0, p.bank.tau, p.bank.n, p.T0)
            s2.define_sky(p.nhat)
            return s2.search(k)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        n_e2e = max(1, min(3, args.steps))
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, dist, f"cuda:{dev}")
        e2e = {"value": job_rate(world, U, n_e2e, dt), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": n_e2e}
        s2.close()

    # roofline of the dominant kernel (group_kernel): ALU-issue bound
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    kern_ms = statistics.mean(kernel_ms)
    achieved = U / (kern_ms / 1000.0)
    clock_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = sm_count * 128 * clock_mhz * 1e6 / 2.0      # 2 lane-ops per lookup
    traffic = group_kernel_traffic(U)
    roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Glookup/s",
            "frac": achieved / peak, "traffic": traffic,
            "kernel": "group_kernel", "kernel_ms": kern_ms,
            "peak_basis": f"{sm_count} SMs x 128 lanes x {clock_mhz:.0f} MHz / 2 lane-ops per lookup"}
    l2_gbps = None
    try:
        l2_gbps = tcw.probe_read_bandwidth(64 << 20, passes=50, reps=5)
    except Exception:
        l2_gbps = None
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        peaks = {}
    hbm = float(peaks.get("hbm_gbs", 6782.8))
    fma = {}
    try:
        fma = {"fp64_tflops": tcw.probe_fma_rate(True), "fp32_tflops": tcw.probe_fma_rate(False),
               "basis": "8 independent fma chains per thread, 8 x 256 threads per SM, best of 5"}
    except Exception as exc:
        fma = {"error": f"{type(exc).__name__}: {exc}"}
    # share of the evaluated lookups that add nothing (segment before T0, bin out of
    # band): from W1 of a search of a sample of the bank (unit weights: W1 counts the
    # valid lookups of a pair)
    invalid = None
    if rank == 0 and p.weights is None and len(p.bank) >= 2048:
        try:
            import tcw_synth as syn
            sub = syn.rng(7).choice(len(p.bank), 2048, replace=False)
            s3 = tcw.Search(dev, stream=stream)
            s3.set_option(tcw.OPT_KEEP_STATS, 1)
            s3.load_problem(p)
            s3.define_bank(p.bank.f0[sub], p.bank.tau[sub], p.bank.n[sub], p.T0)
            s3.search(k)
            w1 = s3.statistics(("W1",))["W1"]
            s3.close()
            D, Nseg = p.rho.shape[:2]
            invalid = {"share": float(1.0 - w1.astype(np.float64).mean() / (D * Nseg)),
                       "sample": f"2048 random templates of the bank x {S} skies (W1 of unit weights)"}
        except Exception as exc:
            invalid = {"error": f"{type(exc).__name__}: {exc}"}
    gather = {"algorithmic_GBps": achieved * p.rho.itemsize / 1e9,
              "measured_l2_read_GBps": l2_gbps,
              "frac_of_measured_l2": (achieved * p.rho.itemsize / 1e9 / l2_gbps) if l2_gbps else None,
              "frac_of_measured_hbm": achieved * p.rho.itemsize / (hbm * 1e9),
              "basis": "4 B per lookup (fp32 map) / read bandwidth of the library's streaming "
                       "probe over a 64 MiB L2-resident buffer, measured in this run"}

    extras = {}
    if rank == 0 and world == 1 and args.workload == "full" and not args.no_amplitude:
        # the same search with the Eq. 3 amplitude weight (f(t_j)/f0)^4 on every
        # lookup, with the number count (rho > 1.6) in place of the power, and
        # with two-bin lookups
        def variant(name, on, off, meta):
            try:
                on()
                s.search(k, psi_out, idx_out)      # warm-up (builds the count bit map)
                torch.cuda.synchronize()
                v_ms = []
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                n_v = max(1, min(3, args.steps))
                a0.record(stream)
                for _ in range(n_v):
                    s.search(k, psi_out, idx_out)
                    v_ms.append(s.info().search_ms)
                a1.record(stream)
                torch.cuda.synchronize()
                ms = a0.elapsed_time(a1) / n_v
                extras[name] = dict(meta, value=U / (ms / 1000.0), unit=UNIT, ms_per_step=ms,
                                    kernel_ms=statistics.mean(v_ms), steps=n_v,
                                    vs_plain=(U / (ms / 1000.0)) / value)
            except Exception as exc:
                extras[name] = {"error": f"{type(exc).__name__}: {exc}"}
            finally:
                off()

        # the same data searched with a device-generated uniform random bank of the
        # same size and box (streamed in 2^18-template chunks, running top-k), and
        # the generation rate of a 1e8-template range written to device memory
        try:
            f_hi = p.f_min + p.rho.shape[2] * p.df
            gspec = tcw.bank_spec(tcw.BANK_RANDOM, (p.f_min, 3500.0, 3.0), (f_hi, 35000.0, 7.0),
                                  n_tmpl=len(p.bank), seed=20250712)
            s.search_generated(gspec, p.T0, k, psi_out, idx_out)          # warm-up
            torch.cuda.synchronize()
            g_ms = []
            for _ in range(max(1, min(2, args.steps))):
                s.search_generated(gspec, p.T0, k, psi_out, idx_out)
                g_ms.append(s.generated_info()["total_ms"])
            gi = s.generated_info()
            n_gen = 10**8
            bufs = tuple(torch.empty(n_gen, dtype=torch.float64, device=f"cuda:{dev}") for _ in range(3))
            big = tcw.bank_spec(tcw.BANK_RANDOM, (500.0, 3500.0, 3.0), (3000.0, 35000.0, 7.0), n_tmpl=10**9,
                                seed=1)
            s.generate_bank(big, 0, n_gen, out=bufs)
            torch.cuda.synchronize()
            t_g = time.perf_counter()
            s.generate_bank(big, 10**9 - n_gen, n_gen, out=bufs)
            torch.cuda.synchronize()
            gen_rate = n_gen / (time.perf_counter() - t_g)
            del bufs
            gms = statistics.mean(g_ms)
            extras["generated"] = {"value": U / (gms / 1000.0), "unit": UNIT, "ms_per_step": gms,
                                   "search_ms": gi["search_ms"], "chunks": gi["chunks"],
                                   "chunk_templates": gi["chunk_templates"], "vs_plain": (U / (gms / 1000.0)) / value,
                                   "bank": "uniform random (Philox), same size and box as the plain bank",
                                   "generate_templates_per_s": gen_rate,
                                   "generate_sample": f"{n_gen} templates (f0, tau, n) of a 1e9-template bank, "
                                                      f"written to device memory, host-timed"}
        except Exception as exc:
            extras["generated"] = {"error": f"{type(exc).__name__}: {exc}"}
        s.define_bank(p.bank.f0, p.bank.tau, p.bank.n, p.T0)      # the plain bank again
        torch.cuda.empty_cache()

        variant("amplitude", lambda: s.set_option(tcw.OPT_AMPLITUDE_POWER, 4),
                lambda: s.set_option(tcw.OPT_AMPLITUDE_POWER, 0), {"amp_power": 4})
        variant("number_count", lambda: s.set_statistic(tcw.STAT_NUMBER_COUNT, 1.6),
                lambda: s.set_statistic(tcw.STAT_POWER), {"rho_th": 1.6})
        variant("two_bin", lambda: s.set_option(tcw.OPT_TRACK_BINS, 2),
                lambda: s.set_option(tcw.OPT_TRACK_BINS, 1), {"track_bins": 2})

        # the precision form: the same workload with the map stored in FP16
        # (fp32 accumulation), and the change of S against the fp32 map on a
        # 2048-template sample
        try:
            rho16 = p.rho.astype(np.float16)
            s16 = tcw.Search(dev, stream=stream)
            s16.load_spectrogram(rho16, p.f_min, p.df, p.t_mid, p.weights)
            s16.load_velocity(p.velocity)
            s16.define_bank(p.bank.f0, p.bank.tau, p.bank.n, p.T0)
            s16.define_sky(p.nhat)
            s16.search(k, psi_out, idx_out)
            torch.cuda.synchronize()
            h0 = torch.cuda.Event(enable_timing=True)
            h1 = torch.cuda.Event(enable_timing=True)
            n16 = max(1, min(3, args.steps))
            h0.record(stream)
            for _ in range(n16):
                s16.search(k, psi_out, idx_out)
            h1.record(stream)
            torch.cuda.synchronize()
            ms16 = h0.elapsed_time(h1) / n16
            import tcw_synth as syn
            sub = syn.rng(11).choice(len(p.bank), 2048, replace=False)
            svals = []
            for ctx in (s, s16):
                ctx.set_option(tcw.OPT_KEEP_STATS, 1)
                ctx.define_bank(p.bank.f0[sub], p.bank.tau[sub], p.bank.n[sub], p.T0)
                ctx.search(k)
                svals.append(ctx.statistics(("S",))["S"].astype(np.float64))
                ctx.set_option(tcw.OPT_KEEP_STATS, 0)
            s.define_bank(p.bank.f0, p.bank.tau, p.bank.n, p.T0)
            s16.close()
            ok = svals[0] > 0
            rel = np.abs(svals[1] - svals[0])[ok] / svals[0][ok]
            extras["fp16"] = {"value": U / (ms16 / 1000.0), "unit": UNIT, "ms_per_step": ms16, "steps": n16,
                              "vs_plain": (U / (ms16 / 1000.0)) / value,
                              "s_rel_change_vs_fp32_map": {"max": float(rel.max()),
                                                           "rms": float(np.sqrt(np.mean(rel ** 2))),
                                                           "sample": "2048 templates x all skies"}}
        except Exception as exc:
            extras["fp16"] = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and args.workload == "full":
        for name, fn, skip in (("small", bench_small, False),
                               ("batched", bench_batched, args.no_batched),
                               ("learned", bench_learned, args.no_learned),
                               ("batched_learned", bench_batched_learned,
                                args.no_learned or args.no_batched)):
            if skip:
                continue
            try:
                extras[name] = fn(args, dev)
            except Exception as exc:   # keep the headline line even if a form fails
                extras[name] = {"error": f"{type(exc).__name__}: {exc}"}
            torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "full":
        rate, threads, n, dt = oracle_rate(p, args.cpu_seconds)
        D, Nseg, _ = p.rho.shape
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{n} random (sky, template) pairs x {D} detectors x {Nseg} segments "
                         f"({n * D * Nseg:.3g} lookups, {dt:.1f} s)",
               "cpu": cpu_model()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": p.name, "global_batch": world * S * len(p.bank),
                       "seq_len": int(p.rho.shape[1]), "parallelism": f"sky-sharded x{world}",
                       "detectors": int(p.rho.shape[0]), "bins": int(p.rho.shape[2]),
                       "templates": len(p.bank), "skies_per_gpu": int(S), "topk": k,
                       "l2": "inputs larger than L2 (power map 800 MB)",
                       "kernel": {1: "group", 2: "lookup"}.get(info.kernel, "?")},
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "gather": gather,
            "cpu_baseline": cpu, "clocks": clocks,
            "search": {"general_path_lanes": info.general_path_lanes,
                       "doppler_bins_max": info.doppler_bins_max, "quantum": info.quantum,
                       "invalid_lookups": invalid},
            "fma_rate": fma,
        }
        line.update(extras)
        print(json.dumps(line))
    s.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return bench_reference(args)
    return bench_ours(args)


if __name__ == "__main__":
    sys.exit(main())
