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
  cpu_baseline  the serial CPU oracle (one core) on one sweep of an
                L = 16384 lattice (256 MiB, streamed from host DRAM), plus
                a cache-resident L = 2048 sample and one oracle instance
                per host core (aggregate).
  u4            the same workload in the packed 4-bit layout.
  q15_u8, q15_u4, q96_u8
                the other paper-scale configurations: q = 15 at L = 32768
                (both layouts) and q = 96 at L = 16384, at the same three
                temperatures, device-timed.
  mid           the L = 4096 heating and cooling ladders (41 temperatures,
                2000 sweeps each), updates/s.
  heatbath      the same workload with the heat-bath update rule.
  fused         the same workload under the fused sweep schedule (both
                colour passes in one kernel, 2 bytes per spin per sweep).
  batched       the 256-lattice batched configuration.
  served        the first 200 requests of the served stream at 200 req/s
                (offered load above capacity: latency measures the backlog);
  served_subcap the same requests arriving at the rate that offers about
                0.8 of the measured served throughput (latency measures
                service);
  served_full   the whole 10000-request stream at 200 req/s.

With --gpus N > 1 under torchrun (one rank per GPU) the paper-scale lattice
is split into N row strips, one per rank, with the halo rows exchanged by
NCCL before every colour pass and the counts all-reduced after every sweep
(strong scaling); the time is the max over ranks.  --gpus N without torchrun
splits it over N devices of this process.
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
KERNEL_SOURCES = ["pass_u8.cuh", "pass_u4.cuh", "philox.cuh", "kernels.cu"]


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
U4_FULLSET_FILE = os.path.join(ROOT, "profiles",
                               "colour_pass_u4_L16384_q9.md")


def instructions_per_site(path=FULLSET_FILE):
    """Thread instructions per updated site of the white and black passes
    from a committed full-set ncu summary (the ALU check beside the HBM
    roofline); None when the kernel sources changed since the capture."""
    try:
        text = open(path).read()
    except OSError:
        return None
    mh = re.search(r"Kernel sources hash:\s*([0-9a-f]+)", text)
    mi = re.search(r"warp instructions \|[^|]*\(([0-9.]+) per updated site\) \|"
                   r"[^|]*\(([0-9.]+) per site\)", text)
    if not (mh and mi) or mh.group(1) != kernel_hash():
        return None
    return {"white": float(mi.group(1)), "black": float(mi.group(2)),
            "source": f"profiles/{os.path.basename(path)} (ncu, L = 16384)"}


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


# ------------------------------------------------------- row strips
def run_strips_ranks(args):
    """N > 1 under torchrun, one rank per GPU: the paper-scale lattice
    (L = 32768, q = 9, seed 11) split into N row strips, strip r on rank r;
    before each colour pass neighbouring ranks exchange one halo row (NCCL
    send/receive), after each sweep the (1 + q) counts are summed
    (all-reduce).  Strong scaling: the whole job is one lattice; value =
    time per spin update of the whole lattice, max over ranks."""
    import numpy as np
    import torch

    from paper_1101_0876_gb300 import potts, strips, workloads
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    init_dist(ws, "nccl")
    cfg = workloads.PAPER_Q9
    L, q = args.L or cfg.L, cfg.q
    N = L * L
    row0, nrows = strips.partition(L, ws)[rank]
    band = strips.StripBand(L, q, potts.START_RANDOM, cfg.seed, row0, nrows,
                            device=local)
    sw = strips.StripSweeper(band, rank, ws)
    betas = [workloads.beta_at(q, t) for t in cfg.t_over_tc]
    K, W = args.steps, args.warmup
    seg = [K // 3 + (1 if k < K % 3 else 0) for k in range(3)]
    recs = torch.zeros((max(K, 1), 1 + q), dtype=torch.int64, device=dev)
    for _ in range(W):
        sw.sweep(betas[0])
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(ws)
    torch.cuda.synchronize(dev)
    st = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    k = 0
    for b, n in zip(betas, seg):
        for _ in range(n):
            sw.sweep(b, record=recs[k])
            k += 1
    e1.record(st)
    torch.cuda.synchronize(dev)
    dev_ms = e0.elapsed_time(e1)
    barrier(ws)
    dev_ms_max = reduce_max(dev_ms, ws, dev)
    # end to end: one sweep per step, its record read back to the host
    barrier(ws)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for b, n in zip(betas, seg):
        for _ in range(n):
            sw.sweep(b).cpu()
    e2e_s = time.perf_counter() - t0
    barrier(ws)
    e2e_max = reduce_max(e2e_s, ws, dev)
    clocks.stop()
    B_last = int(recs[K - 1, 0].item())
    band.close()
    if rank != 0:
        return None
    hbm, kind = measured_peaks()
    pass_ms = dev_ms_max / (2 * K)
    bytes_per_launch = 1.5 * nrows * L
    achieved = bytes_per_launch / (pass_ms * 1e-3) / 1e9
    return {
        "metric": METRIC, "value": dev_ms_max * 1e6 / (N * K), "unit": UNIT,
        "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": dev_ms_max / K, "higher_is_better": False,
        "scaling": "strong", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (random start from Philox, seed 11)",
        "config": {"workload": f"paper_scale_L{L}_q{q}_u8", "L": L, "q": q,
                   "start": "random", "seed": cfg.seed,
                   "t_over_tc": list(cfg.t_over_tc),
                   "parallelism": f"row_strips{ws}",
                   "strip_rows": nrows,
                   "exchange": "one halo row per neighbour and colour pass "
                               "(NCCL send/recv), (1+q) counts all-reduced "
                               "per sweep",
                   "l2": "no flush: each strip's planes exceed L2 at N <= 8"},
        "updates_per_s": N * K / (dev_ms_max * 1e-3),
        "e2e": {"value": e2e_max * 1e9 / (N * K), "unit": UNIT,
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": (1 + q) * 8},
        "gpu_launches": 2 * K,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                     "peak_source": f"{kind} hbm_gbs",
                     "kernel": "colour pass of one strip (per GPU), halo "
                               "exchange and all-reduce included in the "
                               "time", "bytes_per_launch": bytes_per_launch},
        "last_bonds": B_last,
        "clocks": clocks.summary(),
    }


def run_strips_local(args):
    """--gpus N without torchrun: the paper-scale lattice split into N row
    strips on devices 0..N-1 of this one process (potts_create_sharded; halo
    rows by device-to-device copies).  Needs N visible devices."""
    import torch

    from paper_1101_0876_gb300 import potts, workloads
    n = int(args.gpus)
    have = torch.cuda.device_count()
    if have < n:
        raise SystemExit(f"--gpus {n} without torchrun needs {n} visible "
                         f"devices, found {have}")
    cfg = workloads.PAPER_Q9
    L, q = args.L or cfg.L, cfg.q
    N = L * L
    lat = potts.Lattice(L, q, potts.START_RANDOM, cfg.seed, nstrips=n,
                        devices=list(range(n)))
    betas = [workloads.beta_at(q, t) for t in cfg.t_over_tc]
    K, W = args.steps, args.warmup
    seg = [K // 3 + (1 if k < K % 3 else 0) for k in range(3)]
    lat.sweep(betas[0], W, records=False)
    for d in range(n):
        torch.cuda.synchronize(d)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    t0 = time.perf_counter()
    for b, k in zip(betas, seg):
        lat.sweep(b, k)
    secs = time.perf_counter() - t0
    clocks.stop()
    lat.close()
    return {
        "metric": METRIC, "value": secs * 1e9 / (N * K), "unit": UNIT,
        "n_gpus": n, "steps": K, "warmup": W, "ms_per_step": secs * 1e3 / K,
        "higher_is_better": False, "scaling": "strong", "vs_baseline": None,
        "dtype": "u8", "data": "synthetic (random start from Philox, seed 11)",
        "config": {"workload": f"paper_scale_L{L}_q{q}_u8", "L": L, "q": q,
                   "parallelism": f"row_strips{n} (one process)"},
        "updates_per_s": N * K / secs,
        "e2e": {"value": secs * 1e9 / (N * K), "unit": UNIT,
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": (1 + q) * 8},
        "gpu_launches": 2 * n * K,
        "timing": "wall clock around potts_sweep (records to host)",
        "clocks": clocks.summary(),
    }


# --------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    from paper_1101_0876_gb300 import potts, workloads

    ws, rank, local = dist_env()
    if ws > 1:
        return run_strips_ranks(args)
    if args.gpus > 1:
        return run_strips_local(args)
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
    # one call per temperature (the records of its sweeps come back to the
    # host at the end of the call), an event at every boundary: the
    # per-temperature times are reported beside the total
    parts = [(b, n) for b, n in zip(betas, seg) if n > 0]
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
               "get_spins download, amortised per step: the 1 GiB upload and "
               "download are a fixed cost, so this figure depends on K (it "
               "approaches e2e as K grows)"}

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
                    "note": "the timed steps in three consecutive parts "
                            "(one potts_sweep call per temperature, records "
                            "to host at the end of each), CUDA events "
                            "between parts"},
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic (random start from Philox, seed 11 + rank)",
        "config": {"workload": f"paper_scale_L{L}_q{q}_u8",
                   "L": L, "q": q, "start": "random", "seed": cfg.seed,
                   "t_over_tc": list(temps), "sweeps_per_step": 1,
                   "l2": "no flush: 2 GiB of planes per sweep > 126 MB L2",
                   "parallelism": "single GPU"},
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
    if not args.no_u4:
        lat.close()
        line["u4"] = measure_config(args, L, q, potts.LAYOUT_U4, temps,
                                    max(10, args.steps))
        line["u4"]["inst_per_site"] = instructions_per_site(U4_FULLSET_FILE)
    if not args.no_configs:
        lat.close()
        c15, c96 = workloads.PAPER_Q15, workloads.PAPER_Q96
        n_t = max(10, args.steps)   # sweeps per temperature and call
        line["q15_u8"] = measure_config(args, c15.L, c15.q, potts.LAYOUT_U8,
                                        c15.t_over_tc, n_t)
        line["q15_u4"] = measure_config(args, c15.L, c15.q, potts.LAYOUT_U4,
                                        c15.t_over_tc, n_t)
        line["q96_u8"] = measure_config(args, c96.L, c96.q, potts.LAYOUT_U8,
                                        c96.t_over_tc, n_t)
        line["mid"] = measure_mid(args)
    if not args.no_heatbath:
        lat.close()
        line["heatbath"] = measure_heatbath(args, L, q, betas)
    if not args.no_fused:
        lat.close()
        line["fused"] = measure_fused(args, L, q, betas, ns)
    if not args.no_batched:
        lat.close()
        line["batched"] = measure_batched(args, line["updates_per_s"])
    if not args.no_served:
        lat.close()
        line["served"] = measure_served(args, line["updates_per_s"])
        # below capacity: arrivals at the rate that offers ~0.8 of the
        # throughput the saturated server just delivered
        cap = line["served"]["updates_per_s"]
        per_req = (line["served"]["offered_updates_per_s"]
                   / args.served_rate)
        rate = 0.8 * cap / per_req
        line["served_subcap"] = measure_served(
            args, line["updates_per_s"], rate=rate)
        if not args.no_served_full:
            line["served_full"] = measure_served(
                args, line["updates_per_s"], n=10000, rate=args.served_rate)
    if not args.no_cpu_baseline:
        Lc = args.cpu_L_dram
        nsu, dt = cpu_oracle_ns_per_update(Lc, q, betas[1], 1, cfg.seed)
        line["cpu_baseline"] = {
            "value": nsu, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"serial oracle, one sweep of an L={Lc} q={q} lattice "
                      f"(random start, T_c; {Lc * Lc // 2**20} MiB, larger "
                      f"than the host's caches; {dt:.1f} s)"}
        Lc, sweeps = args.cpu_L, args.cpu_sweeps
        nsu, dt = cpu_oracle_ns_per_update(Lc, q, betas[1], sweeps, cfg.seed)
        line["cpu_baseline"]["cache_resident"] = {
            "value": nsu, "unit": UNIT, "cores": 1,
            "sample": f"serial oracle, L={Lc} q={q} ({Lc * Lc // 2**20} "
                      f"MiB) random start at T_c, {sweeps} sweeps "
                      f"({dt:.1f} s)"}
        ups, ncores, wall = cpu_oracle_all_cores(512, q, betas[1],
                                                 args.cpu_sweeps_all, cfg.seed)
        line["cpu_baseline"]["all_cores"] = {
            "value": 1e9 / ups, "unit": UNIT, "updates_per_s": ups,
            "cores": ncores,
            "sample": f"{ncores} independent serial oracles (one process "
                      f"per core), each L=512 q={q} random start at T_c, "
                      f"{args.cpu_sweeps_all} sweeps ({wall:.1f} s)"}
    return line


# -------------------------------------------- single-lattice configurations
def measure_config(args, L, q, layout, t_over_tc, sweeps_per_t, seed=11):
    """One paper-scale configuration (random start, seed 11): sweeps_per_t
    sweeps at each temperature in turn, device-timed with CUDA events per
    temperature; the lattice exceeds L2, so no flush is needed."""
    import torch
    from paper_1101_0876_gb300 import potts, workloads
    stream = torch.cuda.Stream()
    lat = potts.Lattice(L, q, potts.START_RANDOM, seed, layout=layout)
    lat.set_stream(stream.cuda_stream)
    betas = [workloads.beta_at(q, t) for t in t_over_tc]
    lat.sweep(betas[0], 3, records=False)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(betas) + 1)]
    torch.cuda.synchronize()
    evs[0].record(stream)
    for b, ev in zip(betas, evs[1:]):
        lat.sweep(b, sweeps_per_t)
        ev.record(stream)
    torch.cuda.synchronize()
    ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(len(betas))]
    lat.close()
    N = L * L
    bpu = 1.5 if layout == potts.LAYOUT_U4 else 3.0
    tot = sum(ms)
    n = sweeps_per_t * len(betas)
    hbm, kind = measured_peaks()
    gbs = bpu * N * n / (tot * 1e-3) / 1e9
    return {"value": tot * 1e6 / (N * n), "unit": UNIT, "L": L, "q": q,
            "layout": "u4" if layout == potts.LAYOUT_U4 else "u8",
            "t_over_tc": list(t_over_tc), "sweeps_per_t": sweeps_per_t,
            "ns_per_update_per_t": [x * 1e6 / (N * sweeps_per_t) for x in ms],
            "updates_per_s": N * n / (tot * 1e-3),
            "bytes_per_update": bpu, "achieved_gbs": gbs,
            "frac_hbm": gbs / hbm, "peak_source": f"{kind} hbm_gbs"}


def measure_mid(args):
    """The mid configuration (L = 4096, q = 9): heating from the ordered
    start and cooling from the random start over 41 temperatures in
    [0.97, 1.03] T_c, 2000 sweeps each, seed 7, records formed every sweep
    (FP64 e and m on the host).  The 16 MiB lattice stays in L2, so the
    figure is updates/s, not an HBM fraction."""
    from paper_1101_0876_gb300 import protocol, workloads
    cfg = workloads.MID
    L, q = cfg["L"], cfg["q"]
    temps = [workloads.tc(q) * t for t in cfg["ladder"]]
    n = args.mid_sweeps
    heat = protocol.ladder(L, q, temps, 0, n, 1, protocol.START_ORDERED,
                           cfg["seed"])
    cool = protocol.ladder(L, q, temps[::-1], 0, n, 1, protocol.START_RANDOM,
                           cfg["seed"])
    secs = heat[1] + cool[1]
    upd = heat[2] + cool[2]
    return {"value": secs * 1e9 / upd, "unit": UNIT,
            "updates_per_s": upd / secs, "seconds": secs, "L": L, "q": q,
            "temperatures": len(temps), "sweeps_per_t": n,
            "timing": "wall clock around the heating and cooling runs "
                      "(potts_sweep per temperature, records to host)",
            "heating_e_at_tc": heat[0][len(temps) // 2]["e"],
            "cooling_e_at_tc": cool[0][len(temps) // 2]["e"]}


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


def measure_served(args, single_updates_per_s, n=None, rate=None):
    """The served configuration: the first n (default `served_requests`)
    requests of the Poisson stream (`rate` req/s, default 200; L
    log-uniform in [128, 8192]; q in {6, 9, 15, 24, 96}; T in [0.97, 1.03]
    T_c; nsweeps in [100, 5000]; seed = request id), submitted at their
    arrival times to a continuous-batching server with a 120 GB budget;
    latency = time the last record was polled - arrival time."""
    from paper_1101_0876_gb300 import potts, workloads
    n = args.served_requests if n is None else int(n)
    rate = args.served_rate if rate is None else float(rate)
    reqs = workloads.served(n=n, rate_hz=rate)
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
            "rate_hz": rate, "policy": args.served_policy,
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
    ap.add_argument("--cpu-L-dram", type=int, default=16384,
                    help="lattice of the one-sweep CPU oracle sample that "
                         "streams from host DRAM")
    ap.add_argument("--cpu-sweeps", type=int, default=40)
    ap.add_argument("--cpu-sweeps-all", type=int, default=300,
                    help="sweeps per core of the all-cores oracle baseline")
    ap.add_argument("--ref-L", type=int, default=1024)
    ap.add_argument("--no-u4", action="store_true")
    ap.add_argument("--no-heatbath", action="store_true")
    ap.add_argument("--no-fused", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-served-full", action="store_true",
                    help="skip the full 10000-request served stream")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the q=15, q=96 and mid configurations")
    ap.add_argument("--mid-sweeps", type=int, default=2000)
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
