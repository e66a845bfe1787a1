#!/usr/bin/env python3
"""Throughput of the per-time-step vehicle update (vehicle-steps/s) on one B300.

A step is one simulation step of the whole hot path -- sort/merge by lane and position,
neighbour search, IDM + randomized MOBIL, signal stop lines, ballistic advance, lane
transfer, departures, metrics -- over every active vehicle of the workload.

Default workload (city5m): an irregular city -- Delaunay triangulation of 20,000 points in a
30 x 30 km box, 1-4 lanes per edge by length quartile, signals at nodes of degree >= 3 --
with 5,000,000 vehicles on the network and heavy-tailed trip lengths (Pareto 1.5, 1 km,
truncated at 40 km).  Its working set (~400 MB) is far above the 126 MB L2; L2 is still
flushed (256 MiB write) before every timed step, and each step is timed alone with CUDA
events on the simulation's stream.  --workload grid1m: the 100x100 signalised grid, 3 lanes
per direction, 300 m links, 1,000,000 vehicles on the network plus 800,000 gravity-OD trips
departing over 500 s (its ~100 MB working set fits in L2, hence the flush).  Inputs are
generated from a seed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica with its own seed: the step
has no data-path exchange, so the job's time is the slowest rank's and its work the sum.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

KERNELS = ("k_decide", "k_lanes", "k_bucket", "k_apply")
# algorithmic bytes of each kernel: SoA fields it must read / write per vehicle
# (x, v, v0, lane, rp, nxt, id = 28 B), per lane (counts, starts, queue heads), per mover
STEP_LAUNCHES = 5   # k_decide, two lane-scan passes, k_bucket, k_apply
METRICS_BYTES = 56  # ms_read_metrics without the per-lane arrays copies the step control record (56 B)
B_DECIDE_VEH = 48   # reads the 36-B state (x, v, v0, lane, rp, plan word, nl, id); writes x', v', code
B_APPLY_VEH = 72    # reads code, x', v', v0, rp, plan word, nl, id; writes the 36-B state
B_LANES_LANE = 40
B_BUCKET_VEH = 4     # streams the 4-byte result code of every vehicle
B_BUCKET_MOVER = 36  # per arrival: x, x', id, slot reads + the 16-B bucket record


def reduce_over_ranks(total_ms: float, units: float, device: str):
    """Replicas: the job's time is the slowest rank's, its work the sum over ranks."""
    import torch
    import torch.distributed as dist
    mx = torch.tensor([total_ms], dtype=torch.float64, device=device)
    sm = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[0])


def workload(name: str, seed: int):
    from paper_2405_12520_b300 import synth
    if name == "small":   # the small plain-method configuration (reference arm and tests)
        net, dem = synth.small_grid_workload(seed)
        return net, dem, ("4x4 grid, 2 lanes/direction, 200 m links, fixed-time signals; 500 trips "
                          "with uniform OD edges departing over 600 s")
    if name == "grid1m":
        net = synth.large_grid_network()
        # 1M vehicles on the network at t = 0 plus a Poisson inflow of gravity-OD trips
        # that replaces the arrivals, so about 1M stay active over the run
        dem = synth.merge_demands(synth.place_vehicles(net, 1_000_000, seed=seed),
                                  synth.gravity_trips(net, 800_000, t_span=500, seed=seed + 100))
        desc = ("large grid 100x100, 3 lanes/direction, 300 m links, green-wave fixed-time signals; "
                "1,000,000 vehicles pre-placed + 800,000 gravity-OD trips departing over 500 s "
                "(Poisson), v0~N(13.9,1.5)")
    elif name == "city5m":
        net = synth.delaunay_network(20000, box=30000.0, seed=seed)
        dem = synth.place_vehicles(net, 5_000_000, seed=seed, min_spacing=7.0, dest="pareto")
        desc = ("irregular city: Delaunay of 20k points in 30x30 km, 1-4 lanes by length quartile, "
                "signals at degree>=3; 5,000,000 vehicles pre-placed (steady state), heavy-tailed trip "
                "lengths: destination = the one of 256 zones whose shortest-path distance is closest to "
                "a Pareto(1.5, 1 km) draw truncated at 40 km")
    else:
        raise SystemExit(f"unknown workload {name}")
    return net, dem, desc


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def kernel_src_hash() -> str:
    """Hash of every file that shapes the step's kernels and their launches: the kernel
    sources, the host runtime that sizes grids and caps registers, and the build flags."""
    from paper_2405_12520_b300 import build as bld
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_2405_12520_b300")
    files = [os.path.join(pkg, "csrc", f) for f in bld.SOURCES + bld.HEADERS]
    files += [os.path.join(ROOT, "include", "moss103.h"), os.path.join(pkg, "build.py")]
    for f in files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def traffic_per_unit(kernel: str, wl: str):
    """DRAM bytes per vehicle of a kernel from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_src_hash()
    for line in open(path):
        f = line.split("#", 1)[0].split()
        if len(f) == 4 and f[0] == kernel and f[1] == wl and f[3] == src:
            return float(f[2])
    return None


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons around a timed region: sampling
    starts (and the first sample is waited for) before the region, and continues until a
    sample after its end, so a region shorter than the sampling period is still bracketed."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, index: int):
        self.index = index
        self.p = None
        self.rows = []          # (perf_counter time, csv line)
        self.t0 = self.t1 = None

    def _read(self):
        for line in self.p.stdout:
            self.rows.append((time.perf_counter(), line))

    def __enter__(self):
        import threading
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
            deadline = time.perf_counter() + 10.0
            while not self.rows and time.perf_counter() < deadline and self.p.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.p = None
        self.t0 = time.perf_counter()
        return self

    def __exit__(self, *a):
        self.t1 = time.perf_counter()
        if self.p is not None:
            deadline = self.t1 + 2.0
            while (not self.rows or self.rows[-1][0] <= self.t1) and time.perf_counter() < deadline \
                    and self.p.poll() is None:
                time.sleep(0.01)
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        """Samples from the last one before the region's start to the first one after its end."""
        rows = []
        for ts, line in list(self.rows):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                rows.append((ts, float(f[0]), float(f[1]), f[4:8]))
            except ValueError:
                continue
        if not rows or self.t0 is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        lo = max([i for i, r in enumerate(rows) if r[0] <= self.t0] or [0])
        hi = min([i for i, r in enumerate(rows) if r[0] > self.t1] or [len(rows) - 1])
        win = rows[lo:hi + 1]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for *_, fl in win for n, v in zip(names, fl) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in win), "sm_max_mhz": max(r[2] for r in win),
                "reasons": reasons, "samples": len(win), "region_s": round(self.t1 - self.t0, 3),
                "period_ms": self.PERIOD_MS}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def variant(args, net, dem):
    """Model parameters and lane modifications of the run: the default rule set, or the
    max-pressure signals / threshold jitter / lane limits and closures the flags ask for."""
    import numpy as np
    from paper_2405_12520_b300 import synth
    params = synth.default_params(mobil_th_jitter=args.th_jitter,
                                  signal_mode=1 if args.signals == "mp" else 0, mp_interval=args.mp_interval)
    mods, desc = None, {}
    if args.signals == "mp":
        desc["signals"] = f"max pressure, decisions every {args.mp_interval} s"
    if args.th_jitter > 0:
        desc["mobil_th_jitter"] = args.th_jitter
    if args.lane_mods > 0:
        rng = np.random.default_rng(args.seed + 77)
        lim = np.nonzero(rng.random(net.n_lanes) < args.lane_mods)[0].astype(np.int32)
        shut = np.nonzero(rng.random(net.n_lanes) < args.lane_mods / 10)[0].astype(np.int32)
        mods = (lim, rng.uniform(8.0, 14.0, lim.size).astype(np.float32), shut, None)
        desc["lane_mods"] = f"{lim.size} lanes limited to U[8,14] m/s, {shut.size} closed"
    if args.closed_links > 0:
        m = synth.closable_link_masks(net, dem, np.random.default_rng(args.seed + 78), args.closed_links)
        lanes = np.array(list(m), np.int32)
        masks = np.array([m[int(l)] for l in lanes], np.uint32)
        n_all = int(np.diff(net.succ_off)[lanes].sum())
        n_closed = n_all - sum(bin(int(x)).count("1") for x in masks)
        lim, vmax, shut = (mods[:3] if mods is not None else (np.zeros(0, np.int32), np.zeros(0, np.float32),
                                                               np.zeros(0, np.int32)))
        mods = (lim, vmax, shut, (lanes, masks))
        desc["lane_links"] = f"{n_closed} of {n_all} lane links closed, every route still lane-connected"
    return params, mods, desc


def apply_mods(side, mods):
    """Lane limits and closures, then lane links; returns the seconds the calls took."""
    t0 = time.perf_counter()
    if mods is not None:
        lim, vmax, shut, links = mods
        if len(lim):
            side.set_lane_limits(lim, vmax=vmax)
        if len(shut):
            side.set_lane_limits(shut, closed=[1] * len(shut))
        if links is not None:
            side.set_lane_links(*links)
    return time.perf_counter() - t0


def cpu_baseline(net, dem, params, budget_s: float = 12.0, max_steps: int = 60, mods=None, warmup: int = 1,
                 threads: int = 1):
    """The FP64 oracle, as it stands, on this host's cores (threads: its update phase on
    that many OpenMP threads; results identical for any count), on the same workload:
    vehicle-steps/s over up to max_steps steps or budget_s seconds after `warmup` untimed
    steps."""
    import oracle
    o = oracle.Oracle(net, dem, params, threads=threads)
    apply_mods(o, mods)
    for _ in range(warmup):
        o.step()
    n_act = int((o.state()["status"] == 1).sum())
    vs, steps, el = 0, 0, 0.0
    while steps < max_steps and el < budget_s:
        ts = time.perf_counter()
        o.step()
        el += time.perf_counter() - ts
        vs += n_act
        steps += 1
        n_act = int((o.state()["status"] == 1).sum())
    return vs / el, steps, el


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2405_12520_b300 import synth
    net, dem, desc = workload(args.workload, args.seed)
    p, mods, vdesc = variant(args, net, dem)
    k = max(1, min(args.steps, args.ref_steps))
    cores = host_cores()
    val, steps, el = cpu_baseline(net, dem, p, budget_s=1e9, max_steps=k, mods=mods, warmup=args.warmup,
                                  threads=cores)
    line = {
        "impl": "reference", "metric": "vehicle-steps/s", "value": val, "unit": "vehicle-steps/s",
        "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "description": desc, **vdesc},
        "cpu_baseline": {"value": val, "unit": "vehicle-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{steps} oracle steps (update phase on {cores} OpenMP threads) of the "
                                   f"full {args.workload} workload ({dem.n} vehicles) after {args.warmup} "
                                   f"warm-up steps"},
        "e2e": {"value": val, "unit": "vehicle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def full_sort_alternative(sim, stream, flush, avg_ms, reps: int = 20):
    """The non-incremental alternative to the lane merge (k_bucket + k_apply): re-sort the
    whole state by (lane, x) every step with a library radix sort (torch.sort, stable, on
    64-bit keys lane << 32 | bits(x); x > 0, so its bits order like its values) and gather
    the 36-B state by the permutation.  Measured on the current state, L2 flushed, CUDA
    events; a comparison, not a path the simulation uses."""
    import torch
    n = sim.read_metrics(lanes=False)["n_active"]
    x = torch.empty(n, device="cuda")
    v = torch.empty_like(x)
    lane = torch.empty(n, dtype=torch.int32, device="cuda")
    vid = torch.empty_like(lane)
    n = sim.read_state_device(x, v, lane, vid)
    torch.cuda.synchronize()
    keys = (lane.to(torch.int64) << 32) | x.view(torch.int32).to(torch.int64)
    # the other state arrays (v0, rp, nl: 4 B; link plan: 8 B) stand in by same-sized copies
    cols = [x, v, x.clone(), lane, lane.clone(), lane.clone(), vid, keys.clone()]
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    t_sort = t_all = 0.0
    for r in range(reps + 3):
        flush.zero_()
        e0.record(stream)
        sk, perm = torch.sort(keys, stable=True)
        e1.record(stream)
        out = [c.index_select(0, perm) for c in cols]
        e2.record(stream)
        e2.synchronize()
        if r >= 3:
            t_sort += e0.elapsed_time(e1)
            t_all += e0.elapsed_time(e2)
        del out
    ordered = bool(torch.equal(sk, keys))   # the state is already in this order
    return {"what": "torch.sort (stable) of the (lane, x) keys + gather of 36 B/vehicle",
            "vehicles": int(n), "sort_us": round(1e3 * t_sort / reps, 2),
            "sort_and_gather_us": round(1e3 * t_all / reps, 2),
            "merge_us": round(1e3 * (avg_ms[2] + avg_ms[3]), 2), "state_already_sorted": ordered}


def run_ours(args):
    import numpy as np
    import torch
    from paper_2405_12520_b300 import moss, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    net, dem, desc = workload(args.workload, args.seed + rank)
    params, mods, vdesc = variant(args, net, dem)
    stream = torch.cuda.current_stream()
    sim = moss.Sim(params, stream=stream, n_windows=1, block=args.block)
    sim.load_network(net)
    sim.add_vehicles(dem)
    mod_s = apply_mods(sim, mods)
    if mods is not None and mods[3] is not None:
        vdesc["lane_links_call_s"] = round(mod_s, 3)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    sim.step(args.warmup)
    sim.sync()
    n_act = [sim.read_metrics(lanes=False)["n_active"]]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    n_act_steps = []
    with Clocks(local) as clk:
        for k in range(args.steps):
            n_act_steps.append(sim.read_metrics(lanes=False)["n_active"])   # synchronises
            flush.zero_()
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
        barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    n_end = sim.read_metrics(lanes=False)["n_active"]
    # active vehicles at the start of each timed step (read between steps, outside the
    # timed region: the events bracket the step alone)
    per_step = n_act_steps
    vsteps = float(sum(per_step))
    total_ms = float(sum(ms))
    if world > 1:
        total_ms, vsteps = reduce_over_ranks(total_ms, vsteps, "cuda")
    value = vsteps / (total_ms * 1e-3)

    # per-kernel device time (kernel-by-kernel launches, L2 flushed before each step)
    prof_steps = min(args.steps, 50)
    kms = np.zeros(4)
    n0 = sim.read_metrics(lanes=False)["n_active"]
    movers = 0
    for _ in range(prof_steps):
        flush.zero_()
        kms += sim.step_timed(1)
        movers += sim.read_metrics(lanes=False)["movers"]
    n1 = sim.read_metrics(lanes=False)["n_active"]
    n_avg = 0.5 * (n0 + n1)
    units = {"k_decide": n_avg * B_DECIDE_VEH, "k_lanes": net.n_lanes * B_LANES_LANE,
             "k_bucket": n_avg * B_BUCKET_VEH + movers / prof_steps * B_BUCKET_MOVER,
             "k_apply": n_avg * B_APPLY_VEH}
    avg_ms = kms / prof_steps
    dom = KERNELS[int(np.argmax(avg_ms))]
    hbm, src = peaks()
    ach = units[dom] / (avg_ms[KERNELS.index(dom)] * 1e-3) / 1e9
    tpu = traffic_per_unit(dom, args.workload)
    per_unit = net.n_lanes if dom == "k_lanes" else n_avg
    roofline = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None if tpu is None else tpu * per_unit, "kernel": dom,
                "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback 6400 GB/s",
                "kernel_ms": dict(zip(KERNELS, [round(x, 5) for x in avg_ms])),
                # each kernel's algorithmic bytes over its own time, as a fraction of the peak
                "kernel_frac": {k: round(units[k] / (avg_ms[i] * 1e-3) / 1e9 / hbm, 4)
                                for i, k in enumerate(KERNELS) if avg_ms[i] > 0},
                "algorithmic_bytes": {"k_decide": f"{B_DECIDE_VEH} B/vehicle", "k_apply": f"{B_APPLY_VEH} B/vehicle",
                                      "k_lanes": f"{B_LANES_LANE} B/lane",
                                      "k_bucket": f"{B_BUCKET_VEH} B/vehicle + {B_BUCKET_MOVER} B/arrival"},
                "step_effective_gbs": n_avg * (B_DECIDE_VEH + B_APPLY_VEH) / (avg_ms.sum() * 1e-3) / 1e9}
    full_sort = full_sort_alternative(sim, stream, flush, avg_ms)

    # end to end through the public API, wall clock: every step ms_step(1) and a read of the
    # step's result on the host -- its counters (vehicles active, inserted, arrived, summed
    # travel time, device error bits: ms_read_metrics without the per-lane arrays, which
    # waits for the step)
    e2e_steps = min(args.steps, 50)
    barrier()
    t0 = time.perf_counter()
    e2e_vs = 0
    for k in range(e2e_steps):
        n_k = sim.read_metrics(lanes=False)["n_active"]   # vehicles the next step advances
        sim.step(1)
        e2e_vs += n_k
    m_end = sim.read_metrics(lanes=False)
    t1 = time.perf_counter()
    assert m_end["err"] == 0
    e2e = {"value": e2e_vs / (t1 - t0), "unit": "vehicle-steps/s", "h2d_bytes_per_step": 0,
           "d2h_bytes_per_step": METRICS_BYTES,
           "what": "ms_step(1) + ms_read_metrics (step counters: active, inserted, arrived, summed travel "
                   "time, error bits) into host memory every step, wall clock"}
    # the same with the whole per-vehicle state (x, v, lane, id: 16 B/vehicle) exported into
    # pinned host buffers every step (Sec. III-A: position and speed of every vehicle each
    # step), the export of each step running on a side stream while the next step computes
    # (ms_read_state_async / ms_read_wait, two pinned buffer sets used in turn)
    cap = dem.n
    bufs = [dict(x=torch.empty(cap, dtype=torch.float32, pin_memory=True),
                 v=torch.empty(cap, dtype=torch.float32, pin_memory=True),
                 lane=torch.empty(cap, dtype=torch.int32, pin_memory=True),
                 vid=torch.empty(cap, dtype=torch.int32, pin_memory=True)) for _ in range(2)]
    barrier()
    t0 = time.perf_counter()
    x_vs = 0
    d2h = 0
    sim.read_state_async(**bufs[0])
    for k in range(e2e_steps):
        sim.step(1)
        sim.read_state_async(**bufs[(k + 1) % 2])   # queued behind the export in flight
        n_k, _ = sim.read_wait()          # the state step k advanced, now on the host
        x_vs += n_k
        d2h += 16 * n_k
    n_k, _ = sim.read_wait()
    d2h += 16 * n_k
    t1 = time.perf_counter()
    e2e_state = {"value": x_vs / (t1 - t0), "unit": "vehicle-steps/s", "h2d_bytes_per_step": 0,
                 "d2h_bytes_per_step": int(d2h / e2e_steps),
                 "what": "ms_step(1) + ms_read_state_async/ms_read_wait of x, v, lane, id into pinned host "
                         "buffers every step (two exports queued, overlapping the steps), wall clock; bound "
                         "by the host link"}
    sim.sync()

    line = {
        "metric": "vehicle-steps/s", "value": value, "unit": "vehicle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "gpu_launches": (STEP_LAUNCHES + (1 if args.signals == "mp" else 0)) * args.steps,
        "config": {"workload": args.workload, "description": desc, **vdesc, "vehicles": dem.n,
                   "lanes": net.n_lanes, "active_start": n_act[0], "active_end": n_end,
                   "l2": "flushed (256 MiB write) before every timed step; each step timed alone",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline, "e2e": e2e, "e2e_state_export": e2e_state, "clocks": clk.summary(),
        "full_sort_alternative": full_sort,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, steps, el = cpu_baseline(net, dem, params, mods=mods)
        cores = host_cores()
        val_n, steps_n, el_n = cpu_baseline(net, dem, params, mods=mods, threads=cores)
        line["cpu_baseline"] = {"value": val, "unit": "vehicle-steps/s", "cores": 1, "kind": "oracle",
                                "sample": f"{steps} single-threaded FP64 oracle steps of the same workload "
                                          f"({dem.n} vehicles), {el:.1f} s",
                                "all_cores": {"value": val_n, "unit": "vehicle-steps/s", "cores": cores,
                                              "sample": f"{steps_n} FP64 oracle steps, update phase on {cores} "
                                                        f"OpenMP threads (bit-identical to one), {el_n:.1f} s"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.destroy()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batch(args):
    """256 independent scenarios of uneven size: one batched simulation (disjoint union,
    launch shapes from the autotuner, CUDA-graph replays) vs 256 separate simulations each
    stepped with its own ms_step on the same stream."""
    import numpy as np
    import torch
    from paper_2405_12520_b300 import moss, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    n_scen = args.scenarios
    t0 = time.perf_counter()
    sc = synth.batch_scenarios(n_scen, seed=args.seed + 1000 * rank, n_lanes=3, link_len=300.0)
    gen_s = time.perf_counter() - t0
    nets, dems = [n for n, _ in sc], [d for _, d in sc]
    params = synth.default_params()
    stream = torch.cuda.current_stream()

    def vehicle_steps(t_arr, n, t_first, k):
        arr = np.sort(t_arr[t_arr > 0])
        return float(sum(n - int(np.searchsorted(arr, t_first + j, side="right")) for j in range(k)))

    # batched
    b = moss.Sim(params, stream=stream)
    b.load_network_batch(nets)
    b.add_vehicles_batch(dems)
    tune_ms, tune_cfg = b.autotune(trial_steps=3)
    b.step(args.warmup)
    b.sync()
    t_first = b.read_metrics(lanes=False)["t"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        e0.record(stream)
        b.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    st = b.read_state()
    vs_b = vehicle_steps(st["t_arr"], b.n_trips, t_first, args.steps)
    m_b = b.read_metrics(lanes=False)
    b.destroy()
    # separate
    sims = []
    for n, d in sc:
        s = moss.Sim(params, stream=stream)
        s.load_network(n)
        s.add_vehicles(d)
        s.step(args.warmup)
        sims.append(s)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        for s in sims:
            s.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    vs_s = 0.0
    for s in sims:
        st_s = s.read_state()
        vs_s += vehicle_steps(st_s["t_arr"], s.n_trips, t_first, args.steps)
        s.destroy()
    value = vs_b / (ms_b * 1e-3)
    line = {
        "metric": "vehicle-steps/s", "value": value, "unit": "vehicle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "gpu_launches": STEP_LAUNCHES * args.steps,
        "config": {"workload": "batch256", "scenarios": n_scen, "vehicles": int(sum(d.n for d in dems)),
                   "lanes": int(sum(n.n_lanes for n in nets)),
                   "description": "grids 4x4..32x32, 3 lanes, 300 m links, random signal plans; vehicles per "
                                  "scenario log-uniform in [500, 200k] (capped at 60% of jam capacity), pre-placed",
                   "l2": "inputs larger than L2; steps timed back to back", "generation_s": round(gen_s, 1)},
        "autotune": {"best_ms_per_step": tune_ms, "block": tune_cfg[0], "decide_grid_factor": tune_cfg[1],
                     "apply_grid_factor": tune_cfg[2], "lane_scan_threads_per_tile": tune_cfg[3],
                     "bucket_block": tune_cfg[4], "bucket_grid_factor": tune_cfg[5],
                     "searched": "27 (block 128/256/512 x decide, apply grid factor 1/2/4), then lane-scan "
                                 "threads per 1024-lane tile 128/256/512, then bucket block 128/256/512 x "
                                 "grid factor 1/2: 36 trials of 3 steps"},
        "separate": {"value": vs_s / (ms_s * 1e-3), "ms_per_step": ms_s / args.steps,
                     "gpu_launches": STEP_LAUNCHES * n_scen * args.steps},
        "speedup_vs_separate": (vs_b / ms_b) / (vs_s / ms_s),
        "errors": m_b["err"], "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def mlp_grad_us(x, y, cw, batch=8192, reps=200):
    """Device time of one minibatch gradient (operand packing, clearing, the training kernel,
    scaling) with each training kernel, CUDA events over reps calls after a warm-up."""
    import torch
    from paper_2405_12520_b300 import learned, moss
    th = torch.tensor(learned.init_params(3), device="cuda")
    work = torch.zeros(moss.MLP_WORK_FLOATS, device="cuda")
    g = torch.zeros_like(th)
    idx = torch.arange(min(batch, x.shape[0]), dtype=torch.int32, device="cuda")
    out = {}
    for name, tc in (("tcgen05", True), ("mma_sync", False)):
        for _ in range(5):
            moss.mlp_grad(x, y, idx, th, cw, work, g, tc=tc)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            moss.mlp_grad(x, y, idx, th, cw, work, g, tc=tc)
        e1.record()
        torch.cuda.synchronize()
        out[name] = round(1e3 * e0.elapsed_time(e1) / reps, 2)
    return out


def run_learned(args):
    """Learned lane-change surrogate on the large grid: trained on decisions logged from
    small-grid runs of the rule-based step, then timed against the rule-based step on the
    same 1M-vehicle workload (L2 flushed before every timed step)."""
    import numpy as np
    import torch
    from paper_2405_12520_b300 import learned, moss, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    params = synth.default_params()
    t0 = time.perf_counter()
    # training data: decisions logged by the rule-based step on the small 4x4 grid (500
    # trips; denser seeds for standing queues; runs starting in a jam), 256 scenarios per
    # batched simulation, until train_samples are logged
    x, y, runs = learned.collect_batched(learned.mixed_specs(args.train_scenarios), params, 3600,
                                         args.train_samples)
    t_collect = time.perf_counter() - t0
    cw, cnt = learned.class_weights(y)
    grad_us = mlp_grad_us(x, y, cw)   # one gradient call of each kernel (also their first launches)
    theta, info = learned.train(x, y, epochs=args.train_epochs, batch=8192, lr=2e-3, seed=1, class_w=cw)
    # the same training on the mma.sync kernel
    _, info_mma = learned.train(x, y, epochs=args.train_epochs, batch=8192, lr=2e-3, seed=1, class_w=cw, tc=False)
    if args.workload == "learned5m":   # the same network at 5M vehicles (near jam density)
        net = synth.large_grid_network()
        dem = synth.place_vehicles(net, 5_000_000, seed=args.seed, min_spacing=6.0)
        desc = ("large grid 100x100, 3 lanes/direction, 300 m links, green-wave fixed-time signals; "
                "5,000,000 vehicles pre-placed (fronts >= 6 m apart), gravity-OD routes, v0~N(13.9,1.5)")
    else:
        net, dem, desc = workload("grid1m", args.seed)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for name in ("rule", "learned"):
        sim = moss.Sim(params, stream=stream, n_windows=1)
        sim.load_network(net)
        sim.add_vehicles(dem)
        if name == "learned":
            sim.set_lc_model(theta, 0.2)
        sim.step(args.warmup)
        sim.sync()
        if name == "learned":
            sim.set_lc_model(theta, 0.2)   # resets the counters: count the timed steps only
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        nact = []
        for k in range(args.steps):
            nact.append(sim.read_metrics(lanes=False)["n_active"])
            flush.zero_()
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        m = sim.read_metrics()
        out[name] = dict(value=sum(nact) / (ms * 1e-3), ms_per_step=ms / args.steps,
                         mean_speed=float(m["vsum"].sum() / max(1, m["vcnt"].sum())), err=m["err"])
        if name == "learned":
            st = sim.read_lc_stats()   # before the per-kernel pass below adds to the counters
        kms = np.zeros(4)
        for _ in range(20):   # per-kernel device time (k_decide includes k_learn), L2 flushed
            flush.zero_()
            kms += sim.step_timed(1)
        out[name]["kernel_ms"] = dict(zip(KERNELS, [round(x, 5) for x in kms / 20]))
        if name == "learned":
            out[name]["stats"] = st
            out[name]["agreement"] = st["agree"] / max(1, st["candidates"])
            out[name]["fallback_rate"] = st["fallbacks"] / max(1, st["candidates"])
            for r, rn in enumerate("slr"):
                row = sum(st[f"conf_{rn}{f}"] for f in "slr")
                out[name][f"agree_{rn}"] = st[f"conf_{rn}{rn}"] / max(1, row)
        sim.destroy()
    # per-lane 5-minute mean speeds and trajectories: both rules from the same start over the
    # first 300-step window; speeds compared on lanes with at least 300 vehicle-steps in both
    # runs, trajectories on the trips active in both at the end of the window
    win, fin = {}, {}
    for name in ("rule", "learned"):
        sim = moss.Sim(params, stream=stream, n_windows=1)
        sim.load_network(net)
        sim.add_vehicles(dem)
        if name == "learned":
            sim.set_lc_model(theta, 0.2)
        sim.step(int(params["window"]))
        m = sim.read_metrics()
        win[name] = (m["vsum"][0].astype(np.float64), m["vcnt"][0].astype(np.float64))
        if name == "learned":   # agreement over the whole window (more candidates than the timed steps)
            sw = sim.read_lc_stats()
            out["learned"]["window_agreement"] = {
                "steps": int(params["window"]), "candidates": sw["candidates"],
                "agreement": sw["agree"] / max(1, sw["candidates"]),
                "fallback_rate": sw["fallbacks"] / max(1, sw["candidates"]),
                **{f"agree_{rn}": sw[f"conf_{rn}{rn}"] / max(1, sum(sw[f"conf_{rn}{f}"] for f in "slr"))
                   for rn in "slr"}}
        st = sim.read_state(trips=False)
        lane = np.full(dem.n, -1, np.int64)
        xx = np.zeros(dem.n)
        lane[st["id"]] = st["lane"]
        xx[st["id"]] = st["x"]
        fin[name] = (lane, xx, m["arrived"])
        sim.destroy()
    (gv, gc), (rv, rc) = win["learned"], win["rule"]
    busy = (gc >= 300) & (rc >= 300)
    rel = np.abs(gv[busy] / gc[busy] - rv[busy] / rc[busy]) / np.maximum(rv[busy] / rc[busy], 1e-6)
    lane_err = {"lanes": int(busy.sum()), "mean_rel": float(rel.mean()), "p90_rel": float(np.quantile(rel, 0.9)),
                "window_s": int(params["window"])}
    (la, xa, arr_l), (lb, xb, arr_r) = fin["learned"], fin["rule"]
    both = (la >= 0) & (lb >= 0)
    same = both & (la == lb)
    dx = np.abs(xa[same] - xb[same])
    traj = {"after_steps": int(params["window"]), "trips_active_in_both": int(both.sum()),
            "same_lane_frac": float(same.sum() / max(1, both.sum())),
            "same_lane_mean_abs_dx_m": float(dx.mean()) if dx.size else 0.0,
            "same_lane_p90_abs_dx_m": float(np.quantile(dx, 0.9)) if dx.size else 0.0,
            "arrived_learned": int(arr_l), "arrived_rule": int(arr_r)}
    L = out["learned"]
    line = {
        "metric": "vehicle-steps/s", "value": L["value"], "unit": "vehicle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": L["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 state, bf16 MLP operands / f32 accumulate",
        "data": "synthetic", "gpu_launches": (STEP_LAUNCHES + 1) * args.steps,   # + k_learn
        "config": {"workload": args.workload, "description": desc + "; lane-change decisions by the learned MLP",
                   "l2": "flushed (256 MiB write) before every timed step; each step timed alone",
                   "train": {"samples": int(x.shape[0]), "class_counts": cnt.tolist(), "scenario_runs": runs,
                             "demand_mix": "4x4 grid: 30% 500 trips, 10% 1,500, 10% 3,000, 15% 5,000 "
                                           "(standing queues), 20% 2,500 placed 6 m apart + 500 trips, "
                                           "15% 2,900 placed + 300 trips (jam)",
                             "collect_s": round(t_collect, 1), "epochs": args.train_epochs,
                             "adam_steps": info["steps"], "batch": 8192,
                             "train_s": round(info["seconds"], 2), "class_w": info["class_w"],
                             "kernel": "tcgen05 (k_mlp_train_tc)",
                             "train_s_mma_sync": round(info_mma["seconds"], 2),
                             "grad_call_us": grad_us}},
        "learned": L, "rule": out["rule"],
        "learned_vs_rule": L["value"] / out["rule"]["value"],
        "mean_speed_rel_diff": abs(L["mean_speed"] - out["rule"]["mean_speed"]) / out["rule"]["mean_speed"],
        "lane_mean_speed_error": lane_err, "trajectory_vs_rule": traj,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_small(args):
    """The small grid workload as a whole run: 4x4 grid, 500 trips, 3600 steps, on the GPU
    (CUDA-graph replays, timed with events) and through the oracle (one core).
    vehicle-steps = sum of the trips' travel times (every trip arrives)."""
    import torch
    from paper_2405_12520_b300 import moss, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    net, dem = synth.small_grid_workload(args.seed)
    params = synth.default_params()
    stream = torch.cuda.current_stream()
    runs = []
    for k in range(max(1, min(args.steps, 5)) + args.warmup):
        sim = moss.Sim(params, stream=stream, n_windows=12)
        sim.load_network(net)
        sim.add_vehicles(dem)
        pre = 0   # vehicle-steps of the untimed first 16 steps (these also build the step graphs)
        for _ in range(16):
            pre += sim.read_metrics(lanes=False)["n_active"]
            sim.step(1)
        sim.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(3600 - 16)
        b.record(stream)
        sim.sync()
        m = sim.read_metrics(lanes=False)
        if k >= args.warmup:
            runs.append((a.elapsed_time(b), m, pre))
        sim.destroy()
    ms = sum(r[0] for r in runs) / len(runs)
    m = runs[-1][1]
    assert m["err"] == 0 and m["arrived"] == dem.n
    # all trips arrived: their travel times are the run's vehicle-steps; the timed region
    # holds all but those of the first 16 steps
    vsteps = float(m["sum_tt"] - runs[-1][2])
    line = {
        "metric": "vehicle-steps/s", "value": vsteps / (ms * 1e-3), "unit": "vehicle-steps/s", "n_gpus": world,
        "steps": 3600, "warmup": args.warmup, "ms_per_step": ms / (3600 - 16), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "gpu_launches": STEP_LAUNCHES * (3600 - 16),
        "config": {"workload": "small", "description": "4x4 grid, 2 lanes, 200 m links, 500 trips departing "
                   "over 600 s; one whole 3600-step run per repetition (steps 16..3600 timed, and the "
                   "vehicle-steps they hold)", "repetitions": len(runs)},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        o = oracle.Oracle(net, dem, params, n_windows=12)
        t0 = time.perf_counter()
        o.run(3600)
        el = time.perf_counter() - t0
        om = o.metrics()
        line["cpu_baseline"] = {"value": om["sum_tt"] / el, "unit": "vehicle-steps/s", "cores": 1, "kind": "oracle",
                                "sample": f"the whole 3600-step run, {el:.2f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_whole(args):
    """A whole run at the paper's largest scale: 2,464,950 trips on the 100x100 grid (1M on
    the network at t = 0, the rest departing over the hour), 3600 steps of dt = 1 s through
    ms_step (16-step graphs, no L2 flushes: the production loop), timed with CUDA events;
    vehicle-steps are counted exactly by the lane metrics (every active vehicle of every
    step's snapshot, twelve 300-s windows)."""
    import numpy as np
    import torch
    from paper_2405_12520_b300 import moss, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    n_total, n_placed = 2_464_950, 1_000_000
    net = synth.large_grid_network()
    t0 = time.perf_counter()
    dem = synth.merge_demands(synth.place_vehicles(net, n_placed, seed=args.seed + rank),
                              synth.gravity_trips(net, n_total - n_placed, t_span=3600, seed=args.seed + 100 + rank))
    gen_s = time.perf_counter() - t0
    params = synth.default_params()
    stream = torch.cuda.current_stream()
    sim = moss.Sim(params, stream=stream, n_windows=12)
    sim.load_network(net)
    sim.add_vehicles(dem)
    sim.step(16)   # builds the step graphs; counted in the metrics, not in the time
    sim.sync()
    pre = int(sim.read_metrics()["vcnt"].sum())
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier_t0 = time.perf_counter()
    a.record(stream)
    sim.step(3600 - 16)
    b.record(stream)
    sim.sync()
    wall = time.perf_counter() - barrier_t0
    ms = a.elapsed_time(b)
    m = sim.read_metrics()
    assert m["err"] == 0
    vsteps = float(m["vcnt"].sum()) - pre
    if world > 1:
        ms, vsteps = reduce_over_ranks(ms, vsteps, "cuda")
    line = {
        "metric": "vehicle-steps/s", "value": vsteps / (ms * 1e-3), "unit": "vehicle-steps/s", "n_gpus": world,
        "steps": 3600, "warmup": 16, "ms_per_step": ms / (3600 - 16), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "gpu_launches": STEP_LAUNCHES * (3600 - 16),
        "config": {"workload": "run2m", "description": "100x100 grid, 3 lanes, 300 m links, green-wave plans; "
                   "2,464,950 trips: 1,000,000 on the network at t = 0 and 1,464,950 gravity-OD trips "
                   "departing over 3600 s (Poisson); one 3600-step run, steps 16..3600 timed",
                   "run_seconds": round(ms * 1e-3, 3), "wall_seconds": round(wall, 3),
                   "vehicle_steps": int(vsteps), "arrived": int(m["arrived"]), "inserted": int(m["inserted"]),
                   "generation_s": round(gen_s, 1), "l2": "not flushed: the production step loop"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_routes(args):
    """Demand generation on the GPU: 800,000 gravity-model trips between 1,024 zone edges of
    the 100x100 grid (attractions LogNormal(0, 1), decay 1 / route distance^2) sampled by
    ms_sample_trips, then routed by ms_route_trips (wall clock through the C ABI, host
    arrays in and out); the CPU reference on a bounded sample."""
    import numpy as np
    import torch
    from paper_2405_12520_b300 import moss, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    net = synth.large_grid_network()
    rng = np.random.default_rng(args.seed + rank)
    n = 800_000
    zones = rng.choice(net.n_edges, 1024, replace=False).astype(np.int32)
    A = rng.lognormal(0.0, 1.0, zones.size).astype(np.float32)
    sim = moss.Sim(synth.default_params())
    sim.load_network(net)
    sim.route_trips(zones[:64], zones[64:128])   # builds the route graph once
    reps = max(1, min(args.steps, 3))
    ts = tr = 0.0
    for r in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o, d, t = sim.sample_trips(zones, A, 2, n, 3600, args.seed + 1000 * r)
        t1 = time.perf_counter()
        off, edges, bad = sim.route_trips(o, d)
        t2 = time.perf_counter()
        ts += t1 - t0
        tr += t2 - t1
    ts, tr = ts / reps, tr / reps
    # the radiation model on the same zones (populations = the attractions), sampling only
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ro, rd, rt = sim.sample_trips_radiation(zones, A, n, 3600, args.seed)
    t_rad = time.perf_counter() - t0
    line = {
        "metric": "trips/s", "value": n / (ts + tr), "unit": "trips/s", "n_gpus": world, "steps": reps,
        "warmup": 1, "ms_per_step": 1e3 * (ts + tr), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i64", "data": "synthetic", "gpu_launches": None,
        "config": {"workload": "routes800k", "description": "800,000 gravity trips (1,024 zone edges of the "
                   "100x100 grid, A ~ LogNormal(0,1), gamma 2, departures over 3600 s) sampled by "
                   "ms_sample_trips, then routed by ms_route_trips; one of each per repetition",
                   "sample_ms": 1e3 * ts, "route_ms": 1e3 * tr, "route_edges": int(edges.size),
                   "unreachable": bad, "radiation_sample_ms": 1e3 * t_rad},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        from oracle import routing
        zs, As = zones[:64], A[:64]
        t3 = time.perf_counter()
        so, sd, st = routing.gravity_trips(net, zs, As, 2, 2000, 3600, args.seed, oracle.splitmix64)
        routing.routes(net, so, sd)
        el = time.perf_counter() - t3
        line["cpu_baseline"] = {"value": so.size / el, "unit": "trips/s", "cores": 1, "kind": "oracle",
                                "sample": f"2000 trips between 64 of the zones: sampling + scipy Dijkstra "
                                          f"from each zone + the next-hop walk, {el:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="city5m")
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--ref-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--scenarios", type=int, default=256)
    ap.add_argument("--train-samples", type=int, default=50_000_000, help="learned: logged samples to train on")
    ap.add_argument("--train-scenarios", type=int, default=40_000, help="learned: small-grid runs available")
    ap.add_argument("--train-epochs", type=int, default=8)
    ap.add_argument("--signals", choices=("fixed", "mp"), default="fixed",
                    help="signal control: fixed-time plans or max pressure")
    ap.add_argument("--mp-interval", type=int, default=10, help="steps between max-pressure decisions")
    ap.add_argument("--th-jitter", type=float, default=0.0, help="per-trip MOBIL threshold jitter (m/s^2)")
    ap.add_argument("--lane-mods", type=float, default=0.0,
                    help="fraction of lanes given a speed limit (a tenth as many are closed)")
    ap.add_argument("--closed-links", type=float, default=0.0,
                    help="fraction of lane links closed (dynamic lanes; routes stay connected)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload.startswith("batch"):
        run_batch(args)
    elif args.workload.startswith("learned"):
        run_learned(args)
    elif args.workload.startswith("routes"):
        run_routes(args)
    elif args.workload == "small":
        run_small(args)
    elif args.workload == "run2m":
        run_whole(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
