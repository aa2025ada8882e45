#!/usr/bin/env python3
"""Benchmark of the checkerboard Metropolis sweep (one JSON line on rank 0).

Workload (default): the paper-scale single lattice L = 32768 (1.07e9 spins,
1 GiB of uint8 spins), q = 9, random start, seed 11, temperatures
{0.995, 1.000, 1.005} T_c.  One step = one sweep (white pass, black pass
fused with the per-sweep {B, hist} counts, record copied to the host,
FP64 observables updated).  The timed steps are split evenly over the three
temperatures, the spins carrying over (Sec. 3 protocol).

Metric: ns per spin update (time / (N * sweeps)), whole job, lower is better.

  value     device time (CUDA events on the library's stream) of the timed
            sweeps, lattice resident in HBM (2 GiB of planes > 126 MB L2, so
            no L2 flush is needed between steps).
  e2e       the same sweeps issued one potts_sweep() call per step through
            the public API, host buffers, wall clock: includes the launch, the
            device->host copy of each step's record and the host-side FP64
            observables.  beta travels by value in the launch (0 bytes H2D).
  e2e_job   a whole job through the public API: upload of a host lattice
            (pinned) with potts_set_state, the timed sweeps with records, and
            potts_get_spins of the final lattice.
  roofline  the colour-pass kernel against measured HBM bandwidth, 1.5 bytes
            per spin per pass (read own plane, write own plane, read other
            plane once) = 3 bytes per spin per sweep.
  cpu_baseline  the serial CPU oracle on a bounded sample (one core), plus
                one oracle instance per host core (aggregate).
  heatbath      the same workload with the heat-bath update rule.
  fused         the same workload under the fused sweep schedule (both
                colour passes in one kernel, 2 bytes per spin per sweep).

With torchrun (N > 1) each rank sweeps its own replica (weak scaling, no
data-path collective); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ns/spin-update @L=32768 q=9 (frac HBM peak)"
UNIT = "ns/update"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "colour_pass_L32768_q9_traffic.md")
KERNEL_SOURCES = ["pass_u8.cuh", "philox.cuh", "kernels.cu"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1101_0876_gb300", "csrc", f),
                  "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_per_launch(L: int):
    """DRAM bytes per colour-pass launch from the committed ncu summary,
    scaled from its lattice to L by the number of sites; None when the
    kernel sources changed since the capture."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    mh = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    mb = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    ml = re.search(r"capture_L:\s*(\d+)", text)
    if not (mh and mb and ml) or mh.group(1) != kernel_hash():
        return None
    Lc = int(ml.group(1))
    return float(mb.group(1)) * (L * L) / (Lc * Lc)


FULLSET_FILE = os.path.join(ROOT, "profiles", "colour_pass_L16384_q9.md")


def instructions_per_site():
    """Thread instructions per updated site of the white and black passes
    from the committed full-set ncu summary (the ALU check beside the HBM
    roofline); None when the kernel sources changed since the capture."""
    try:
        text = open(FULLSET_FILE).read()
    except OSError:
        return None
    mh = re.search(r"Kernel sources hash:\s*([0-9a-f]+)", text)
    mi = re.search(r"warp instructions \|[^|]*\(([0-9.]+) per updated site\) \|"
                   r"[^|]*\(([0-9.]+) per site\)", text)
    if not (mh and mi) or mh.group(1) != kernel_hash():
        return None
    return {"white": float(mi.group(1)), "black": float(mi.group(2)),
            "source": "profiles/colour_pass_L16384_q9.md (ncu, L = 16384)"}


# GB300 instruction issue: one warp instruction per clock on each of the
# four sub-partitions of an SM, 32 threads, 152 SMs, 2.07 GHz maximum SM clock.
ISSUE_PEAK = 4 * 32 * 152 * 2.07e9   # thread instructions per second


def alu_roofline(sites_per_s: float):
    """The integer-issue roofline of the colour pass: thread instructions
    per second (sites/s x instructions per site, the latter from the
    committed ncu summary, mean of the two passes) against the issue peak."""
    ips = instructions_per_site()
    if ips is None:
        return None
    per_site = 0.5 * (ips["white"] + ips["black"])
    achieved = sites_per_s * per_site
    return {"bound": "alu", "achieved": achieved, "peak": ISSUE_PEAK,
            "unit": "thread instructions/s", "frac": achieved / ISSUE_PEAK,
            "inst_per_site": per_site,
            "peak_source": "4 warp instructions per clock per SM x 32 x 152 "
                           "SMs x 2.07 GHz"}


# ------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}",
                 f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                    "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, n in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(n)
        pw = [float(r[3]) for r in self.rows
              if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows),
                "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def reduce_max(x: float, ws: int, device=None) -> float:
    """Max over ranks (the slowest rank sets the job's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(base: int, rank: int) -> int:
    """Each rank sweeps its own independent replica (weak scaling)."""
    return base + rank


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------ cpu baseline
def cpu_oracle_ns_per_update(L: int, q: int, beta: float, sweeps: int,
                             seed: int):
    import oracle
    lat = oracle.Lattice(L, q, 1, seed)
    lat.sweep(beta, 1, records=False)            # warm caches
    t0 = time.perf_counter()
    lat.sweep(beta, sweeps)
    dt = time.perf_counter() - t0
    return dt * 1e9 / (L * L * sweeps), dt


def _cpu_oracle_worker(a):
    L, q, beta, sweeps, seed = a
    import oracle
    lat = oracle.Lattice(L, q, 1, seed)
    lat.sweep(beta, 1, records=False)
    t0 = time.perf_counter()
    lat.sweep(beta, sweeps)
    return L * L * sweeps, time.perf_counter() - t0


def cpu_oracle_all_cores(L: int, q: int, beta: float, sweeps: int,
                         seed: int):
    """One independent oracle instance per host core (processes started
    with spawn), each sweeping its own L x L lattice; aggregate updates/s
    over the slowest worker's time."""
    import concurrent.futures as cf
    import multiprocessing as mp
    n = os.cpu_count() or 1
    jobs = [(L, q, beta, sweeps, seed + i) for i in range(n)]
    with cf.ProcessPoolExecutor(n, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_cpu_oracle_worker, jobs))
    upd = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return upd / wall, n, wall


# --------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    from paper_1101_0876_gb300 import potts, workloads

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    init_dist(ws, "nccl")
    cfg = workloads.PAPER_Q9
    L, q = args.L or cfg.L, cfg.q
    N = L * L
    seed = replica_seed(cfg.seed, rank)
    temps = cfg.t_over_tc
    betas = [workloads.beta_at(q, t) for t in temps]

    stream = torch.cuda.Stream(device=dev)
    lat = potts.Lattice(L, q, potts.START_RANDOM, seed)
    lat.set_stream(stream.cuda_stream)

    K, W = args.steps, args.warmup
    seg = [K // 3 + (1 if k < K % 3 else 0) for k in range(3)]
    recbuf = torch.empty((max(K, 1), 1 + q), dtype=torch.int64,
                         pin_memory=True).numpy().view(np.uint64)

    # warm-up (untimed)
    lat.sweep(betas[0], W, records=False)
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)

    # ---- device-timed region
    barrier(ws)
    torch.cuda.synchronize(dev)
    # each temperature's steps in two halves, an event at every boundary:
    # the per-part times give a median over six repetitions beside the total
    parts = [(b, h) for b, n in zip(betas, seg) for h in (n // 2, n - n // 2)
             if h > 0]
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(parts) + 1)]
    evs[0].record(stream)
    off = 0
    for (b, n), ev in zip(parts, evs[1:]):
        lat.sweep(b, n, out=recbuf[off:off + n])
        off += n
        ev.record(stream)
    torch.cuda.synchronize(dev)
    dev_ms = evs[0].elapsed_time(evs[-1])
    part_ms = [evs[i].elapsed_time(evs[i + 1]) / n
               for i, (_, n) in enumerate(parts)]
    barrier(ws)
    dev_ms_max = reduce_max(dev_ms, ws, dev)

    # ---- end to end: one public-API call per step, host record buffers
    barrier(ws)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    step = 0
    for b, n in zip(betas, seg):
        for _ in range(n):
            lat.sweep(b, 1, out=recbuf[step:step + 1])
            step += 1
    e2e_s = time.perf_counter() - t0
    barrier(ws)
    e2e_s_max = reduce_max(e2e_s, ws, dev)
    clocks.stop()

    # ---- whole job through the public API (upload, sweeps, download)
    job = None
    if not args.no_job:
        host = torch.empty((L, L), dtype=torch.uint8,
                           pin_memory=True).numpy()
        lat.spins(out=host)
        out = torch.empty((L, L), dtype=torch.uint8, pin_memory=True).numpy()
        barrier(ws)
        t0 = time.perf_counter()
        lat.set_state(host, 10**6)
        off = 0
        for b, n in zip(betas, seg):
            lat.sweep(b, n, out=recbuf[off:off + n])
            off += n
        lat.spins(out=out)
        job_s = reduce_max(time.perf_counter() - t0, ws, dev)
        job = {"value": job_s * 1e9 / (ws * N * K), "unit": UNIT,
               "h2d_bytes_per_step": N / K, "d2h_bytes_per_step":
               N / K + (1 + q) * 8, "note": "set_state upload + K sweeps + "
               "get_spins download, amortised per step"}

    if rank != 0:
        return None

    ns = dev_ms_max * 1e6 / (ws * N * K)
    hbm, peak_kind = measured_peaks()
    launches = 2 * K
    pass_ms = dev_ms / launches
    bytes_per_launch = 1.5 * N
    achieved = bytes_per_launch / (pass_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC,
        "value": ns,
        "unit": UNIT,
        "n_gpus": ws,
        "steps": K,
        "warmup": W,
        "ms_per_step": dev_ms_max / K,
        "repeats": {"n": len(part_ms),
                    "ms_per_step": [round(x, 5) for x in part_ms],
                    "median_ms_per_step": float(np.median(part_ms)),
                    "note": "the timed steps in six consecutive parts (two "
                            "per temperature), CUDA events between parts"},
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic (random start from Philox, seed 11 + rank)",
        "config": {"workload": f"paper_scale_L{L}_q{q}_u8",
                   "L": L, "q": q, "start": "random", "seed": cfg.seed,
                   "t_over_tc": list(temps), "sweeps_per_step": 1,
                   "l2": "no flush: 2 GiB of planes per sweep > 126 MB L2",
                   "parallelism": f"replicas{ws}"},
        "updates_per_s": ws * N * K / (dev_ms_max * 1e-3),
        "e2e": {"value": e2e_s_max * 1e9 / (ws * N * K), "unit": UNIT,
                "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": (1 + q) * 8},
        "e2e_job": job,
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic_per_launch(L),
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "kernel": "colour pass (white; black fused with counts)",
                     "bytes_per_launch": bytes_per_launch,
                     "inst_per_site": instructions_per_site(),
                     "binding": "integer instruction issue, not HBM: "
                                "see roofline_alu"},
        "roofline_alu": alu_roofline(N * K / (dev_ms * 1e-3)),
        "clocks": clocks.summary(),
    }
    if ws == 1 and not args.no_u4:
        lat.close()
        line["u4"] = measure_u4(args, L, q, betas)
    if ws == 1 and not args.no_heatbath:
        lat.close()
        line["heatbath"] = measure_heatbath(args, L, q, betas)
    if ws == 1 and not args.no_fused:
        lat.close()
        line["fused"] = measure_fused(args, L, q, betas, ns)
    if ws == 1 and not args.no_batched:
        lat.close()
        line["batched"] = measure_batched(args, line["updates_per_s"])
    if ws == 1 and not args.no_served:
        lat.close()
        line["served"] = measure_served(args, line["updates_per_s"])
    if not args.no_cpu_baseline and ws == 1:
        Lc, sweeps = args.cpu_L, args.cpu_sweeps
        nsu, dt = cpu_oracle_ns_per_update(Lc, q, betas[1], sweeps, cfg.seed)
        line["cpu_baseline"] = {
            "value": nsu, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"serial oracle, L={Lc} q={q} random start at T_c, "
                      f"{sweeps} sweeps ({dt:.1f} s); per-update cost of the "
                      f"serial raster loop does not depend on L"}
        ups, ncores, wall = cpu_oracle_all_cores(512, q, betas[1],
                                                 args.cpu_sweeps_all, cfg.seed)
        line["cpu_baseline"]["all_cores"] = {
            "value": 1e9 / ups, "unit": UNIT, "updates_per_s": ups,
            "cores": ncores,
            "sample": f"{ncores} independent serial oracles (one process "
                      f"per core), each L=512 q={q} random start at T_c, "
                      f"{args.cpu_sweeps_all} sweeps ({wall:.1f} s)"}
    return line


# ------------------------------------------------- packed 4-bit layout
def measure_u4(args, L, q, betas):
    """The same workload in the packed 4-bit layout (q <= 16): 1.5 bytes
    per site per sweep, device-timed like `value`."""
    import torch
    from paper_1101_0876_gb300 import potts
    stream = torch.cuda.Stream()
    lat = potts.Lattice(L, q, potts.START_RANDOM, 11, layout=potts.LAYOUT_U4)
    lat.set_stream(stream.cuda_stream)
    lat.sweep(betas[0], 3, records=False)
    n = max(3, args.steps // 2)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lat.sweep(betas[1], n)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lat.close()
    N = L * L
    hbm, _ = measured_peaks()
    gbs = 1.5 * N * n / (ms * 1e-3) / 1e9
    return {"value": ms * 1e6 / (N * n), "unit": UNIT, "sweeps": n,
            "updates_per_s": N * n / (ms * 1e-3),
            "bytes_per_update": 1.5, "achieved_gbs": gbs,
            "frac_hbm": gbs / hbm}


# ------------------------------------------------------ heat-bath rule
def measure_heatbath(args, L, q, betas):
    """The same workload with the heat-bath update (U8), device-timed like
    `value`; same 3 bytes per site per sweep."""
    import torch
    from paper_1101_0876_gb300 import potts
    stream = torch.cuda.Stream()
    lat = potts.Lattice(L, q, potts.START_RANDOM, 11)
    lat.set_update(potts.UPDATE_HEATBATH)
    lat.set_stream(stream.cuda_stream)
    lat.sweep(betas[0], 3, records=False)
    n = max(3, args.steps // 4)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lat.sweep(betas[1], n)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lat.close()
    N = L * L
    hbm, _ = measured_peaks()
    gbs = 3.0 * N * n / (ms * 1e-3) / 1e9
    return {"value": ms * 1e6 / (N * n), "unit": UNIT, "sweeps": n,
            "updates_per_s": N * n / (ms * 1e-3), "achieved_gbs": gbs,
            "frac_hbm": gbs / hbm}


# ------------------------------------------------ fused sweep schedule
def measure_fused(args, L, q, betas, two_pass_ns):
    """The same workload (U8, Metropolis) with both colour passes of a sweep
    in one kernel: each plane read once (plus halos) and written once, 2
    bytes per site per sweep.  Device-timed like `value`."""
    import torch
    from paper_1101_0876_gb300 import potts
    stream = torch.cuda.Stream()
    lat = potts.Lattice(L, q, potts.START_RANDOM, 11, layout=potts.LAYOUT_U8)
    lat.set_schedule(potts.SCHEDULE_FUSED)
    lat.set_stream(stream.cuda_stream)
    lat.sweep(betas[0], 3, records=False)
    n = max(3, args.steps // 2)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lat.sweep(betas[1], n)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lat.close()
    N = L * L
    hbm, _ = measured_peaks()
    gbs = 2.0 * N * n / (ms * 1e-3) / 1e9
    ns = ms * 1e6 / (N * n)
    return {"value": ns, "unit": UNIT, "sweeps": n,
            "updates_per_s": N * n / (ms * 1e-3),
            "bytes_per_update": 2.0, "achieved_gbs": gbs,
            "frac_hbm": gbs / hbm, "vs_two_pass": ns / two_pass_ns,
            "kernel": "fused_sweep_kernel (one launch per sweep)"}


# ------------------------------------------------- batched / served
def measure_batched(args, single_updates_per_s):
    """The batched configuration: 256 lattices (L log-uniform in [64, 2048],
    q in {6, 9, 15, 24}, T in [0.98, 1.02] T_c, seeds 1000 + i) swept
    together; the first call (which autotunes) is a warm-up, the second
    (500 sweeps) is timed end to end through potts_batch_sweep."""
    from paper_1101_0876_gb300 import potts, workloads
    spec = workloads.batched(sweeps=args.batch_sweeps)
    b = potts.Batch(spec.L, spec.q, spec.start, spec.seed)
    b.sweep(spec.beta, 20, records=False)
    t0 = time.perf_counter()
    b.sweep(spec.beta, spec.sweeps)
    dt = time.perf_counter() - t0
    upd = sum(L * L for L in spec.L) * spec.sweeps
    b.close()
    return {"lattices": len(spec.L), "sweeps": spec.sweeps,
            "updates": upd, "seconds": dt, "updates_per_s": upd / dt,
            "ratio_to_single": (upd / dt) / single_updates_per_s,
            "timing": "wall clock around potts_batch_sweep, records to host"}


def measure_served(args, single_updates_per_s):
    """The served configuration, bounded: the first `served_requests`
    requests of the Poisson stream (200 req/s; L log-uniform in
    [128, 8192]; q in {6, 9, 15, 24, 96}; T in [0.97, 1.03] T_c; nsweeps in
    [100, 5000]; seed = request id), submitted at their arrival times to a
    continuous-batching server with a 120 GB budget; latency = time the
    last record was polled - arrival time."""
    from paper_1101_0876_gb300 import potts, workloads
    reqs = workloads.served(n=args.served_requests, rate_hz=args.served_rate)
    srv = potts.Server(hbm_budget_bytes=120 * 10**9,
                       max_slots=args.served_slots,
                       sweeps_per_step=args.served_k,
                       policy=(potts.ADMIT_SMALLEST
                               if args.served_policy == "smallest"
                               else potts.ADMIT_FIFO))
    import numpy as np
    buf = np.empty(8192 * 257, dtype=np.uint64)   # reused by every poll
    t0 = time.perf_counter()
    nxt = 0
    live = {}
    lat = []
    while nxt < len(reqs) or live:
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt].arrival_s <= now:
            r = reqs[nxt]
            rid = srv.submit(r.L, r.q, r.beta, r.nsweeps, r.seed, r.start)
            live[rid] = r
            nxt += 1
        for rid in list(live):
            _, done = srv.poll(rid, max_sweeps=8192, out=buf)
            if done:
                lat.append(time.perf_counter() - t0 - live.pop(rid).arrival_s)
        time.sleep(0.001)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.stop()
    upd = sum(r.L * r.L * r.nsweeps for r in reqs)
    lat_ms = sorted(1e3 * x for x in lat)

    def pct(p):
        return lat_ms[min(len(lat_ms) - 1, int(round(p / 100 * (len(lat_ms) - 1))))]
    busy = wall - reqs[0].arrival_s
    offered = upd / max(reqs[-1].arrival_s, 1e-9)
    return {"requests": len(reqs), "updates": upd,
            "seconds": busy, "updates_per_s": upd / busy,
            "ratio_to_single": (upd / busy) / single_updates_per_s,
            "p50_ms": pct(50), "p99_ms": pct(99), "max_ms": lat_ms[-1],
            "offered_updates_per_s": offered,
            "slots": args.served_slots, "sweeps_per_step": args.served_k,
            "rate_hz": args.served_rate, "policy": args.served_policy,
            "steps": st["steps"],
            "note": ("offered load exceeds capacity: latency grows with the "
                     "backlog (saturated server)")
            if offered > 0.9 * single_updates_per_s
            else "offered load below the single-lattice rate"}


# --------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle as it stands, timed on the host cores, on the same
    workload's metric: each step is one sweep of an L=cpu_L lattice (q=9,
    random start, T around T_c); ns per update."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    from paper_1101_0876_gb300 import workloads
    import oracle
    cfg = workloads.PAPER_Q9
    q = cfg.q
    Lc = args.ref_L
    betas = [workloads.beta_at(q, t) for t in cfg.t_over_tc]
    lat = oracle.Lattice(Lc, q, 1, cfg.seed)
    for k in range(args.warmup):
        lat.sweep(betas[k % 3], 1, records=False)
    t0 = time.perf_counter()
    for k in range(args.steps):
        lat.sweep(betas[k % 3], 1)
    dt = time.perf_counter() - t0
    ns = dt * 1e9 / (Lc * Lc * args.steps)
    sample = (f"serial oracle, L={Lc} q={q} random start, one sweep per "
              f"step over T/T_c in {list(cfg.t_over_tc)}")
    return {
        "impl": "reference", "metric": METRIC, "value": ns, "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": {"workload": f"paper_scale_L{cfg.L}_q{q}_u8",
                                        "sample_L": Lc},
        "cpu_baseline": {"value": ns, "unit": UNIT, "cores": 1,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": ns, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=240)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=0, help="override lattice size")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-job", action="store_true")
    ap.add_argument("--cpu-L", type=int, default=2048)
    ap.add_argument("--cpu-sweeps", type=int, default=40)
    ap.add_argument("--cpu-sweeps-all", type=int, default=300,
                    help="sweeps per core of the all-cores oracle baseline")
    ap.add_argument("--ref-L", type=int, default=1024)
    ap.add_argument("--no-u4", action="store_true")
    ap.add_argument("--no-heatbath", action="store_true")
    ap.add_argument("--no-fused", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--batch-sweeps", type=int, default=500)
    ap.add_argument("--served-requests", type=int, default=200)
    ap.add_argument("--served-slots", type=int, default=64)
    ap.add_argument("--served-policy", choices=["fifo", "smallest"],
                    default="fifo", help="admission order of the server")
    ap.add_argument("--served-rate", type=float, default=200.0,
                    help="Poisson arrival rate of the served stream (req/s)")
    ap.add_argument("--served-k", type=int, default=32)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)
    ws, _, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
