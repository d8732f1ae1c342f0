#!/usr/bin/env python
"""Benchmark of the truncated transforms over Z/(2^32768+1) at L = 2^16 (n swept over
32769, 40000, 45000, 52000, 65536), the workload on which the TFT/ITFT throughput is quoted.

One step = for every n of the sweep, a TFT (Algorithm 1) then an ITFT with the final division
by L (Algorithm 2) on resident device buffers, each n on its own CUDA stream (five independent
problems); the round trip restores the inputs, so every step sees the same data. Per-n times
come from a separate pass that runs the round trips one after another. Throughput counts the algorithmic bytes of the paper's two-pass
Bailey schedule: every cell a top-level row or column sub-transform reads or writes, times
8 (N/64 + 1) bytes per cell (see alg_bytes_tft / alg_bytes_itft), divided by device time.

Prints one JSON line (rank 0). Multi-GPU runs (torchrun) are independent replicas: every
rank runs the whole sweep on its own GPU, no data moves between GPUs, and the value is the
bytes of all ranks divided by the slowest rank's time (weak scaling).

--impl reference times the CPU oracle (the paper's recursion on the host cores) on a bounded
sample of the same workload: one round trip at n = 40000 per step.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "TFT/ITFT GB/s vs HBM peak; batched Z[x] products/s vs plain, bit-exact"
WORKLOAD = workloads.TRANSFORM_LARGE
FALLBACK_HBM_GBS = 6800.0


# ---------------------------------------------------------------- algorithmic bytes
def _split(l):
    l1 = l // 2
    return l1, l - l1


def alg_cells_tft(l, z, n):
    """Cells read + written by the two passes of Algorithm 1's top level (Sec. 3)."""
    _, l2 = _split(l)
    L2 = 1 << l2
    n1p = -(-n // L2)
    z1, z2 = divmod(z, L2)
    z2p = L2 if z1 > 0 else z2
    return (z + n1p * z2p) + (n1p * z2p + n)


def alg_cells_itft(l, z, n, f=0):
    """Cells read + written by the four phases of Algorithm 2's top level (Sec. 4)."""
    _, l2 = _split(l)
    L2 = 1 << l2
    n1, n2 = divmod(n, L2)
    z1, z2 = divmod(z, L2)
    fp = 1 if n2 + f > 0 else 0
    z2p = L2 if z1 > 0 else z2
    m, mp = min(n2, z2), max(n2, z2)
    cells = n1 * 2 * L2  # full rows
    for u in range(n2, z2p):  # rightmost columns
        cells += (z1 + 1 if u < mp else z1) + n1 + fp
    if fp:  # last row
        cells += z2p + n2 + f
    for u in range(n2):  # leftmost columns
        cells += (z1 + 1 if u < m else z1) + n1 + 1
    return cells


def cell_bytes(N):
    return 8 * (N // 64 + 1)


def plan_bytes(tg, kind, l, n, N):
    """Bytes of the cells every job of the plan of one transform call reads (nload) and writes
    (nstore), each cell 8 W bytes (the N + 1 bits, no padding)."""
    try:
        plan = tg.transform_jobs(kind, l, n, n, N, scale=kind)
    except tg.TftError:
        return None
    cells = sum(j["nload"] + j["nstore"] for launch in plan["launches"] for j in launch["jobs"])
    return cells * cell_bytes(N)


def cell_stride(W, requested):
    """Limbs between consecutive cells: W rounded up to even (16-byte aligned cells) unless a
    stride is requested, which must hold a cell (>= W) and keep 16-byte alignment (even)."""
    if not requested:
        return W + (W & 1)
    if requested < W or requested % 2:
        raise SystemExit(f"--stride must be an even number of limbs >= {W}")
    return requested


def step_bytes(N, l, ns):
    return sum((alg_cells_tft(l, n, n) + alg_cells_itft(l, n, n)) * cell_bytes(N) for n in ns)


# ---------------------------------------------------------------- environment
def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0810_3203_gb300", "csrc")
    # the files that decide what the transform kernel does and which launches a plan makes
    for f in ("common.h", "host.h", "plan.cpp", "program.cpp", "ring_warp.cuh", "job_kernel.cuh",
              "transform_kernel.cu", "transform_k32.cu", "transform_fused_k32.cu"):
        h.update(f.encode())
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu summary, if the
    kernels have not changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic_job_kernel_l16_N32768.json")
    try:
        d = json.load(open(p))
        if d.get("kernel_source_hash") == kernel_source_hash():
            return d
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples every 50 ms, each stamped on arrival. Started before the warm-up (the
    tool takes a moment to start); only the samples stamped inside the timed region
    [mark_start(), mark_stop() + one interval] count. If none lands there (a region shorter than
    the interval), the first sample after the region's start is used and flagged."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_S = 0.05

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(int(self.INTERVAL_S * 1000))],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        deadline = time.perf_counter() + 3.0
        while not self.lines and time.perf_counter() < deadline:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark_start(self):
        self.t0 = time.perf_counter()

    def mark_stop(self):
        self.t1 = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        # one more interval, so that a sample taken inside the region has arrived
        time.sleep(self.INTERVAL_S * 1.5)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        t0 = self.t0 if self.t0 is not None else float("-inf")
        t1 = (self.t1 if self.t1 is not None else float("inf")) + self.INTERVAL_S
        inside = [ln for t, ln in self.lines if t0 <= t <= t1]
        note = None
        if not inside:
            after = [ln for t, ln in self.lines if t >= t0]
            inside = after[:1]
            note = "no sample inside the timed region; the first one after its start"
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in inside:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        out = {"sm_mhz": statistics.median(sm) if sm else None,
               "sm_max_mhz": max(smax) if smax else None,
               "reasons": sorted(reasons), "samples": len(sm), "interval_ms": int(self.INTERVAL_S * 1000)}
        if note:
            out["note"] = note
        return out


# ---------------------------------------------------------------- distributed helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(backend):
    import torch.distributed as dist
    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=ws)
    return ws, rank


def max_over_ranks(value, device=None):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def timed_steps(step, steps, warmup, sync, device=None):
    """W untimed steps, then exactly K steps bracketed by barrier + device sync on both sides;
    returns the slowest rank's elapsed seconds."""
    for _ in range(warmup):
        step()
    sync()
    barrier(device)
    sync()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    sync()
    barrier(device)
    sync()
    return max_over_ranks(time.perf_counter() - t0, device)


# ---------------------------------------------------------------- CPU oracle legs
def oracle_roundtrip_seconds(n, N, l):
    import oracle
    x = workloads.residues(WORKLOAD["seed"], n, N, cells=1 << l)
    t0 = time.perf_counter()
    oracle.tft(x, l, n, n, 0, N)
    oracle.itft(x, l, n, n, 0, 0, N)
    return time.perf_counter() - t0


def reference_sample_n(steps, warmup):
    """n of one step of the reference arm: 40000 (the CPU baseline's n) while steps + warmup
    <= 25, else scaled down so the whole run stays near 25 round trips at n = 40000 of oracle
    work (about 1.5 min on 3.4 s round trips), and never below 2048."""
    return max(2048, min(40000, (40000 * 25) // max(1, steps + warmup)))


def _oracle_roundtrip_task(args):
    return oracle_roundtrip_seconds(*args)


def cpu_baseline(N, l, parallel=True):
    """The oracle's round trip at n = 40000 on one host core; with `parallel`, also the same
    round trip as independent problems, one per process on every host core (a spawned pool:
    the parent process has already used the GPU)."""
    n = 40000
    secs = oracle_roundtrip_seconds(n, N, l)
    b = (alg_cells_tft(l, n, n) + alg_cells_itft(l, n, n)) * cell_bytes(N)
    out = {"value": round(b / secs / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": f"one TFT + ITFT round trip at n = {n} (l = {l}, N = {N}), single thread, "
                     f"{secs:.1f} s"}
    if parallel:
        import multiprocessing as mp
        p = max(1, min(os.cpu_count() or 1, 16))  # each process holds a 269 MB buffer
        with mp.get_context("spawn").Pool(p) as pool:
            pool.map(_oracle_roundtrip_task, [(200, 1024, 8)] * p)  # start every worker
            t0 = time.perf_counter()
            pool.map(_oracle_roundtrip_task, [(n, N, l)] * p)
            wall = time.perf_counter() - t0
        out["parallel"] = {"value": round(p * b / wall / 1e9, 4), "unit": "GB/s", "cores": p,
                           "sample": f"{p} independent round trips at n = {n}, one process each, "
                                     f"{wall:.1f} s wall"}
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    N, l = WORKLOAD["N"], WORKLOAD["l"]
    n = reference_sample_n(args.steps, args.warmup)
    secs = []

    def step():
        secs.append(oracle_roundtrip_seconds(n, N, l))

    for _ in range(args.warmup):
        step()
    secs.clear()
    for _ in range(args.steps):
        step()
    # the oracle's own time (the seeded inputs are generated outside it)
    elapsed = sum(secs)
    b = (alg_cells_tft(l, n, n) + alg_cells_itft(l, n, n)) * cell_bytes(N)
    value = b * args.steps / elapsed / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(elapsed / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"TFT+ITFT round trip over Z/(2^32768+1), L = 2^16, n = {n} "
                               "(bounded sample of the n sweep)", "N": N, "l": l, "ns": [n],
                   "seed": WORKLOAD["seed"]},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} round trips at n = {n}, single thread"},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU leg
def run_gpu(args):
    import numpy as np
    import torch

    import paper_0810_3203_gb300 as tg

    ws, rank, local = dist_env()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    dist_init("nccl")
    tg.load()
    N, l, ns = WORKLOAD["N"], WORKLOAD["l"], list(WORKLOAD["ns"])
    W = N // 64 + 1
    stride = cell_stride(W, args.stride)
    L = 1 << l
    stream = torch.cuda.current_stream(device)
    host = {n: workloads.residues(WORKLOAD["seed"], n, N, stride=stride, cells=L) for n in ns}
    dev = {n: torch.from_numpy(host[n].view(np.int64)).to(device) for n in ns}
    torch.cuda.synchronize(device)

    # launch configuration of the ring: the autotuner's pick, on one of the sweep's buffers (the
    # round trips restore it), outside every timed region; --fused pins the launch form first
    # (the tuner keeps it)
    if args.fused >= 0:
        tg.config_set(N, dict(tg.config_get(N), fused=args.fused))
    if args.tma >= 0:
        tg.config_set(N, dict(tg.config_get(N), tma=args.tma))
    tuned = None if args.no_tune else tg.tune(dev[40000 if 40000 in dev else ns[0]], l, 40000 if 40000 in dev else ns[0],
                                              N, stride, reps=2, stream=stream)

    def mk():
        return torch.cuda.Event(enable_timing=True)

    # one step: the round trip of every n, each n on its own stream (independent problems, so
    # the small serial launches of one ITFT and the last waves of every launch overlap with the
    # work of the others); the main stream forks to them and joins them
    lanes = {n: torch.cuda.Stream(device) for n in ns}

    def step():
        fork = torch.cuda.Event()
        fork.record(stream)
        for n in ns:
            s = lanes[n]
            s.wait_event(fork)
            tg.tft_ex(dev[n], l, n, n, N, 0, stride, stream=s)
            tg.itft_ex(dev[n], l, n, n, 0, N, 0, stride, 1, stream=s)
        for n in ns:
            joined = torch.cuda.Event()
            joined.record(lanes[n])
            stream.wait_event(joined)

    def sync():
        torch.cuda.synchronize(device)

    clocks = ClockSampler(local)
    clocks.start()
    # warm-up, then exactly K timed steps between barriers and device syncs
    for _ in range(args.warmup):
        step()
    sync()
    barrier(device)
    sync()
    start, stop = mk(), mk()
    t0 = time.perf_counter()
    clocks.mark_start()
    start.record(stream)
    for k in range(args.steps):
        step()
    stop.record(stream)
    sync()
    clocks.mark_stop()
    barrier(device)
    sync()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    dev_ms = start.elapsed_time(stop)
    elapsed = max_over_ranks(dev_ms / 1e3, device)

    # per-n times (untimed for the value): the same round trips one after another on one
    # stream, CUDA events around each transform call
    per_reps = max(2, args.steps // 2)
    ev = [{n: (mk(), mk(), mk()) for n in ns} for _ in range(per_reps)]
    for k in range(per_reps):
        for n in ns:
            ev[k][n][0].record(stream)
            tg.tft_ex(dev[n], l, n, n, N, 0, stride, stream=stream)
            ev[k][n][1].record(stream)
            tg.itft_ex(dev[n], l, n, n, 0, N, 0, stride, 1, stream=stream)
            ev[k][n][2].record(stream)
    sync()
    per_n = {n: [0.0, 0.0] for n in ns}
    for k in range(per_reps):
        for n in ns:
            per_n[n][0] += ev[k][n][0].elapsed_time(ev[k][n][1]) / per_reps
            per_n[n][1] += ev[k][n][1].elapsed_time(ev[k][n][2]) / per_reps

    # correctness of the timed data: the round trips restore the inputs
    ok = True
    for n in ns:
        back = dev[n].view(-1, stride)[:n, :W].cpu().numpy().view(np.uint64)
        ok &= bool(np.array_equal(back, host[n].reshape(-1, stride)[:n, :W]))

    sb = step_bytes(N, l, ns)
    value = sb * args.steps * ws / elapsed / 1e9
    # the job kernel is the only kernel of the timed region and its launches on the five streams
    # overlap, so its time is the region's device time on this rank
    achieved = sb * args.steps / (dev_ms / 1e3) / 1e9
    peak, peak_kind = measured_peak()
    launches_per_step = sum(tg.transform_plan(0, l, n, n, N)["launches"] + tg.transform_plan(1, l, n, n, N)["launches"]
                            for n in ns)
    # the record was taken on the default layout
    traffic = recorded_traffic() if stride == cell_stride(W, 0) else None

    # end to end through the C ABI with host buffers: per n, H2D of its n input cells from
    # pinned memory, TFT, ITFT, D2H of its n result cells (the other L - n cells of a buffer are
    # the transforms' scratch and stay on the device). The H2D copies run in order on one stream
    # and each n's D2H on a stream of its own, so that no result waits behind another n's; each
    # n's transforms run on its stream of the timed step, so the copies of one n overlap the
    # transforms of the others; a buffer is refilled only after its previous results have left.
    span = {n: n * stride for n in ns}  # limbs of the n cells
    pinned = {n: torch.from_numpy(host[n].view(np.int64)[:span[n]].copy()).pin_memory() for n in ns}
    outp = {n: torch.empty_like(pinned[n]).pin_memory() for n in ns}
    h2d = sum(pinned[n].numel() * 8 for n in ns)
    s_in = torch.cuda.Stream(device)
    s_out = {n: torch.cuda.Stream(device) for n in ns}
    drained = {}

    def e2e_step():
        for n in ns:
            if n in drained:
                s_in.wait_event(drained[n])
            with torch.cuda.stream(s_in):
                dev[n][:span[n]].copy_(pinned[n], non_blocking=True)
            arrived = torch.cuda.Event()
            arrived.record(s_in)
            lanes[n].wait_event(arrived)
            tg.tft_ex(dev[n], l, n, n, N, 0, stride, stream=lanes[n])
            tg.itft_ex(dev[n], l, n, n, 0, N, 0, stride, 1, stream=lanes[n])
            done = torch.cuda.Event()
            done.record(lanes[n])
            s_out[n].wait_event(done)
            with torch.cuda.stream(s_out[n]):
                outp[n].copy_(dev[n][:span[n]], non_blocking=True)
            drained[n] = torch.cuda.Event()
            drained[n].record(s_out[n])

    e2e_secs = timed_steps(e2e_step, max(1, args.steps // 2), 1, sync, device)
    e2e_value = sb * max(1, args.steps // 2) * ws / e2e_secs / 1e9
    for n in ns:
        ok &= bool(np.array_equal(outp[n].numpy().view(np.uint64).reshape(-1, stride)[:n, :W],
                                  host[n].reshape(-1, stride)[:n, :W]))

    # Sec. 6 zero padding (used inside the products): the exact Algorithm 2 ITFT against the ITFT
    # of n rounded up to whole rows of 2^8 cells (no last-row step), same buffers, timing only
    padded = {}
    for n in ns:
        n_pad = -(-n // 256) * 256

        def exact(n=n):
            tg.itft_ex(dev[n], l, n, n, 0, N, 0, stride, 1, stream=stream)

        def pad(n=n, n_pad=n_pad):
            tg.itft_ex(dev[n], l, n_pad, n_pad, 0, N, 0, stride, 1, stream=stream)

        te = timed_steps(exact, 3, 1, sync, device)
        tp = timed_steps(pad, 3, 1, sync, device)
        padded[str(n)] = {"n_padded": n_pad, "exact_ms": round(te / 3 * 1e3, 3), "padded_ms": round(tp / 3 * 1e3, 3),
                          "passes_exact": tg.transform_plan(1, l, n, n, N)["passes"],
                          "passes_padded": tg.transform_plan(1, l, n_pad, n_pad, N)["passes"]}

    sn = sn_leg(tg, device, stream, 10)
    pointwise = pointwise_leg(tg, device, stream)
    e1 = None if args.no_e1 else e1_leg(tg, device, stream)
    small = small_legs(tg, device, stream)
    ok &= small["small_round_trip"]["bit_exact_roundtrip"]
    ok &= sn["bit_exact_roundtrip"]
    batch = None if args.no_batch else batch_leg(tg, device, stream, 2, 3, not args.no_tune)
    ok &= batch is None or batch["bit_exact_vs_plain"]
    serve = None if args.no_serve else serve_leg(tg, device, stream, args.serve_requests, not args.no_tune,
                                                 slots=args.serve_slots)
    ok &= serve is None or serve["bit_exact_vs_plain"]

    if rank != 0:
        return 0 if ok else 1
    cpu = None if args.no_cpu_baseline else cpu_baseline(N, l)
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(elapsed / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "TFT+ITFT round trips over Z/(2^32768+1), L = 2^16, n in "
                               "{32769, 40000, 45000, 52000, 65536}",
                   "N": N, "l": l, "ns": ns, "seed": WORKLOAD["seed"], "stride_limbs": stride,
                   "bytes_per_step": sb, "l2": "inputs larger than L2 (269 MB per buffer)",
                   "streams": "one per n, forked from and joined to the timing stream",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                     "traffic": traffic.get("dram_bytes_per_tft") if traffic else None,
                     "traffic_unit": "DRAM bytes of one TFT call at n = 40000 (ncu), against "
                                     f"{traffic.get('alg_bytes_per_tft') if traffic else None} algorithmic",
                     "plan_bytes": plan_bytes(tg, 0, l, 40000, N),
                     "plan_bytes_unit": "bytes the plan's jobs read and write in one TFT call at n = 40000 "
                                        "(from zx_transform_jobs; stores still dirty in L2 when a launch ends "
                                        "escape the kernel's ncu counters)",
                     "kernel": "job_kernel_stream<32> run with one CTA per job, one tensor copy per cell in "
                               "and out (every launch of the TFT and ITFT calls; the only kernel of the timed "
                               "region, its time the region's device time)"},
        "per_n_ms": {str(n): [round(a, 3), round(b, 3)] for n, (a, b) in per_n.items()},
        "smoothness": {str(n): round((per_n[n][0] + per_n[n][1]) / (per_n[ns[-1]][0] + per_n[ns[-1]][1]), 4)
                       for n in ns},
        "e2e": {"value": round(e2e_value, 2), "unit": "GB/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "bit_exact_roundtrip": ok,
        "wall_s": round(wall, 3),
    }
    line["zero_padded_itft"] = padded
    line["sn"] = sn
    line["pointwise"] = pointwise
    line["e1_sweep"] = e1
    line.update(small)
    if tuned is not None:
        line["tuned_config"] = tuned
    if batch is not None:
        line["batch"] = batch
    if serve is not None:
        line["serve"] = serve
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0 if ok else 1


def tune_rings(tg, device, stream, shapes, enabled, top=4):
    """Run the autotuner for the rings that carry most of the work of these products (the
    heaviest `top` by estimated cells x ring size), each on a scratch buffer of random residues
    at the largest transform length and median product length seen for it."""
    import numpy as np
    import torch

    if not enabled:
        return None
    rings = {}
    for lf, bf, lg, bg in shapes:
        p = tg.zx_plan(lf, bf, lg, bg)
        r = rings.setdefault(p["N"], {"l": 0, "n": [], "work": 0})
        r["l"] = max(r["l"], p["l"])
        r["n"].append(p["n_fft"])
        r["work"] += p["n_fft"] * p["N"]
    out = {}
    for N, r in sorted(rings.items(), key=lambda kv: -kv[1]["work"])[:top]:
        l, n = r["l"], sorted(r["n"])[len(r["n"]) // 2]
        n = min(n, 1 << l)
        W = N // 64 + 1
        stride = W + (W & 1)
        x = torch.from_numpy(workloads.residues(11, n, N, stride=stride, cells=1 << l).view(np.int64)).to(device)
        info = tg.tune(x, l, n, N, stride, reps=1, stream=stream)
        out[str(N)] = {k: info[k] for k in ("ls_max", "ls_c", "max_warps", "split", "best_ms", "default_ms")}
        del x
    torch.cuda.synchronize(device)
    return out


def batch_leg(tg, device, stream, steps, warmup, tune=True):
    """The 512 mixed products (lengths uniform in [200, 20000], coefficient bits uniform in
    [64, 1024]) with operands resident on the device: one zx_mul_batch call per step against
    the same products as 512 zx_mul calls, results compared word for word."""
    import numpy as np
    import torch

    shapes = workloads.batch_shapes()
    seed = workloads.BATCH_MIXED["seed"] * 1000
    items, outs_plain = [], []
    for k, (lf, lg, bits) in enumerate(shapes):
        m = (bits + 63) // 64
        f = workloads.coefficients(seed + 2 * k, lf, bits, m)
        g = workloads.coefficients(seed + 2 * k + 1, lg, bits, m)
        mh = tg.zx_plan(lf, bits, lg, bits)["limbs_h"]
        F = torch.from_numpy(f.view(np.int64)).to(device)
        G = torch.from_numpy(g.view(np.int64)).to(device)
        H = torch.zeros((lf + lg - 1) * mh, dtype=torch.int64, device=device)
        items.append((F, lf, m, G, lg, m, H, mh, False, bits, bits))
        outs_plain.append(torch.zeros_like(H))
    torch.cuda.synchronize(device)
    tuned = tune_rings(tg, device, stream, [(lf, bits, lg, bits) for lf, lg, bits in shapes], tune)

    def batched():
        tg.zx_mul_batch(items, stream=stream)

    def plain():
        for (F, lf, m, G, lg, _, _, mh, sg, b, _), Hp in zip(items, outs_plain):
            tg.zx_mul(F, lf, m, G, lg, m, Hp, mh, sg, b, b, stream=stream)

    def timed(fn, k, w):
        for _ in range(w):
            fn()
        torch.cuda.synchronize(device)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize(device)
        return a.elapsed_time(b) / 1e3 / k

    tb = timed(batched, steps, warmup)
    tp = timed(plain, max(1, steps // 2), 1)
    same = all(torch.equal(it[6], hp) for it, hp in zip(items, outs_plain))
    count = len(items)
    return {"workload": "512 independent Z[x] products, lengths U[200, 20000], coefficient bits U[64, 1024], "
                        "unsigned, seed 4; each product in its own ring",
            "products_per_s": round(count / tb, 2), "plain_products_per_s": round(count / tp, 2),
            "ms_per_batch": round(tb * 1e3, 3), "ms_plain": round(tp * 1e3, 3),
            "speedup_vs_plain": round(tp / tb, 3), "bit_exact_vs_plain": bool(same), "tuned": tuned}


def serve_leg(tg, device, stream, count, tune=True, rates=(2000.0, 500.0), slots=3):
    """Poisson arrivals of products with lengths log-uniform in [2^8, 2^15] and coefficient bits
    log-uniform in [64, 4096], operands resident on the device: the serving loop (continuous
    batching) against the plain path, where each request runs alone with zx_mul once the
    previous one has finished; latency = completion - arrival. The first rate (2000 requests/s,
    the workload's) is above what one GB300 serves, so its latencies include queueing; the second
    (500/s) is below, so its latencies show what batching adds to a request. The same requests
    (shapes and operands) are offered at both rates."""
    import numpy as np
    import torch

    reqs = workloads.serve_requests(count)
    seed = workloads.SERVE_POISSON["seed"] * 1000
    items, plain_out = [], []
    for k, (_, lf, lg, bits) in enumerate(reqs):
        m = (bits + 63) // 64
        f = workloads.coefficients(seed + 2 * k, lf, bits, m)
        g = workloads.coefficients(seed + 2 * k + 1, lg, bits, m)
        mh = tg.zx_plan(lf, bits, lg, bits)["limbs_h"]
        F = torch.from_numpy(f.view(np.int64)).to(device)
        G = torch.from_numpy(g.view(np.int64)).to(device)
        H = torch.zeros((lf + lg - 1) * mh, dtype=torch.int64, device=device)
        items.append((F, lf, m, G, lg, m, H, mh, False, bits, bits))
        plain_out.append(torch.zeros_like(H))
    torch.cuda.synchronize(device)
    base_rate = workloads.SERVE_POISSON["rate"]
    tuned = tune_rings(tg, device, stream, [(lf, bits, lg, bits) for _, lf, lg, bits in reqs], tune)

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(q * len(v)))]

    def one_rate(rate):
        # the generator's arrival times scale as 1 / rate for the same uniform draws
        arrivals = [t * base_rate / rate for t, _, _, _ in reqs]
        for H in [it[6] for it in items] + plain_out:
            H.zero_()
        torch.cuda.synchronize(device)
        with tg.Server(slots=slots) as srv:
            # every request once, untimed: the plans of all shapes are made before either timed
            # run (otherwise the served run would make them and the plain run, after it, reuse them)
            for it in items:
                srv.submit(*it)
            srv.drain(600.0)
            srv.poll(count + 16)
            lat = {}
            t_srv = time.perf_counter()
            ids = {}
            for k, it in enumerate(items):
                while time.perf_counter() - t_srv < arrivals[k]:
                    pass
                ids[srv.submit(*it)] = k
            srv.drain(600.0)
            t_end = time.perf_counter()
            for rid, st, sec in srv.poll(count + 16):
                if st != 0:
                    raise RuntimeError(f"request {rid} failed with status {st}")
                lat[ids[rid]] = sec
            stats = srv.stats()
        served = [lat[k] for k in range(count)]
        plain_lat = []
        t0 = time.perf_counter()
        for k, ((F, lf, m, G, lg, _, _, mh, sg, b, _), Hp) in enumerate(zip(items, plain_out)):
            while time.perf_counter() - t0 < arrivals[k]:
                pass
            tg.zx_mul(F, lf, m, G, lg, m, Hp, mh, sg, b, b, stream=stream)
            torch.cuda.synchronize(device)
            plain_lat.append(time.perf_counter() - t0 - arrivals[k])
        t_plain = time.perf_counter() - t0
        same = all(torch.equal(it[6], hp) for it, hp in zip(items, plain_out))
        return {"products_per_s": round(count / (t_end - t_srv), 2),
                "p50_ms": round(pct(served, 0.5) * 1e3, 3), "p99_ms": round(pct(served, 0.99) * 1e3, 3),
                "plain_products_per_s": round(count / t_plain, 2),
                "plain_p50_ms": round(pct(plain_lat, 0.5) * 1e3, 3),
                "plain_p99_ms": round(pct(plain_lat, 0.99) * 1e3, 3),
                "offered_per_s": round(count / arrivals[-1], 1), "waves": stats["waves"],
                "max_wave_products": stats["max_wave_products"], "max_waves_in_flight": stats["max_waves_in_flight"],
                "arena_peak_gb": round(stats["arena_peak_bytes"] / 1e9, 3),
                "learned_time_scale": round(stats["time_scale"], 3), "bit_exact_vs_plain": bool(same)}

    res = one_rate(rates[0])
    out = {"workload": f"{count} requests, Poisson arrivals at {rates[0]:g}/s, lengths log-uniform [2^8, 2^15], "
                       "coefficient bits log-uniform [64, 4096], unsigned, seed 5"}
    out.update(res)
    for r in rates[1:]:
        sub = one_rate(r)
        sub["workload"] = f"the same requests at {r:g}/s (below what the GPU serves)"
        out[f"at_{int(r)}_per_s"] = sub
        out["bit_exact_vs_plain"] = out["bit_exact_vs_plain"] and sub["bit_exact_vs_plain"]
    out["slots"] = slots
    out["tuned"] = tuned
    return out


def sn_leg(tg, device, stream, steps):
    """Round trips over S[y]/(y^(M/2)+1) (Sec. 5.2 workload shape): TFT then ITFT with the
    division by L at M = 2048 (elements of 1024 coefficients, 8 KB), L = 2^11, n = 2000,
    resident buffer; algorithmic bytes of the paper's two-pass schedule as for Z/(2^N+1)."""
    import numpy as np
    import torch

    w = workloads.SN_TRANSFORM
    M, m, l, n = w["M"], w["m"], w["l"], w["n"]
    L, H = 1 << l, M // 2
    x = workloads.sn_elements(w["seed"], n, M, m, cells=L)
    d = torch.from_numpy(x.view(np.int64)).to(device)

    def step():
        tg.sn_tft(d, l, n, n, M, m, 0, stream=stream)
        tg.sn_itft(d, l, n, n, 0, M, m, 0, scale=1, stream=stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize(device)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        step()
    b.record(stream)
    torch.cuda.synchronize(device)
    sec = a.elapsed_time(b) / 1e3 / steps
    ok = bool(np.array_equal(d.cpu().numpy().view(np.uint64)[:n * H], x[:n * H]))
    cells = alg_cells_tft(l, n, n) + alg_cells_itft(l, n, n)
    gbs = cells * H * 8 / sec / 1e9
    return {"workload": f"S[y]/(y^{H}+1) over Z/mZ, m = 2^40 + 15, L = 2^{l}, n = {n}, pieces of {M // 4} "
                        "coefficients, seed 7", "ms_per_round_trip": round(sec * 1e3, 3),
            "gbs_algorithmic": round(gbs, 2), "bit_exact_roundtrip": ok}


def small_legs(tg, device, stream, reps=50):
    """The small round trip (TFT then ITFT over Z/(2^1024+1), L = 2^8, n = z = 200) timed call
    by call, its bound being latency; and the medium product (3000 x 2500 coefficients of 2000
    bits, ring N = 4096) through zx_mul. Operands resident; medians of CUDA-event times."""
    import numpy as np
    import torch

    def median_ms(fn):
        for _ in range(5):
            fn()
        torch.cuda.synchronize(device)
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        return statistics.median(times)

    w = workloads.ROUNDTRIP_SMALL
    N, l, n = w["N"], w["l"], w["n"]
    W = N // 64 + 1
    x = workloads.residues(w["seed"], n, N, cells=1 << l)
    d = torch.from_numpy(x.view(np.int64)).to(device)
    t_tft = median_ms(lambda: tg.tft(d, l, n, N, stream=stream))
    t_itft = median_ms(lambda: tg.itft(d, l, n, N, stream=stream))
    t_rt = median_ms(lambda: (tg.tft(d, l, n, N, stream=stream), tg.itft(d, l, n, N, stream=stream)))
    # as many ITFTs as TFTs, each ITFT inverting a TFT: the buffer is back to x
    ok = bool(np.array_equal(d.cpu().numpy().view(np.uint64)[:n * W], x[:n * W]))
    p = workloads.PRODUCT_MEDIUM
    bits, lf, lg = p["bits"], p["len_f"], p["len_g"]
    m = (bits + 63) // 64
    F = torch.from_numpy(workloads.coefficients(p["seed"], lf, bits, m).view(np.int64)).to(device)
    G = torch.from_numpy(workloads.coefficients(p["seed"] + 1, lg, bits, m).view(np.int64)).to(device)
    plan = tg.zx_plan(lf, bits, lg, bits)
    mh = plan["limbs_h"]
    H = torch.zeros((lf + lg - 1) * mh, dtype=torch.int64, device=device)
    t_mul = median_ms(lambda: tg.zx_mul(F, lf, m, G, lg, m, H, mh, False, bits, bits, stream=stream))
    return {"small_round_trip": {"workload": f"Z/(2^{N}+1), L = 2^{l}, n = z = {n}, seed {w['seed']}",
                                 "us_tft": round(t_tft * 1e3, 1), "us_itft": round(t_itft * 1e3, 1),
                                 "us_round_trip": round(t_rt * 1e3, 1), "bit_exact_roundtrip": ok},
            "medium_product": {"workload": f"{lf} x {lg} coefficients of {bits} bits, unsigned, seed {p['seed']}; "
                                           f"ring N = {plan['N']}, L = 2^{plan['l']}",
                               "ms_zx_mul": round(t_mul, 4)}}


def e1_leg(tg, device, stream, reps=3):
    """Products shaped like the Sec. 5.1 measurements: f and g of equal length (512 .. 16384 in
    5 % steps), 8000-bit unsigned coefficients (ring N = 16384, as the paper's "about 16000
    bits"). Per length: the zx_mul device time (operands and result resident), and on the
    product's own ring the time of its three transforms truncated (z = length, n = the padded
    output count) against full length (n = L, a plain power-of-two transform)."""
    import numpy as np
    import torch

    w = workloads.SMOOTHNESS_SWEEP
    lengths, v = [], float(w["len_lo"])
    while int(round(v)) <= w["len_hi"]:
        if not lengths or int(round(v)) != lengths[-1]:
            lengths.append(int(round(v)))
        v *= w["step"]
    if lengths[-1] != w["len_hi"]:
        lengths.append(w["len_hi"])
    bits = w["bits"]
    m = (bits + 63) // 64

    def timed(fn):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(device)
        return a.elapsed_time(b) / reps

    rows = []
    for k, n in enumerate(lengths):
        plan = tg.zx_plan(n, bits, n, bits)
        F = torch.from_numpy(workloads.coefficients(w["seed"] + 2 * k, n, bits, m).view(np.int64)).to(device)
        G = torch.from_numpy(workloads.coefficients(w["seed"] + 2 * k + 1, n, bits, m).view(np.int64)).to(device)
        mh = plan["limbs_h"]
        H = torch.empty((2 * n - 1) * mh, dtype=torch.int64, device=device)
        t_mul = timed(lambda: tg.zx_mul(F, n, m, G, n, m, H, mh, False, bits, bits, stream=stream))
        l, N, st, nf = plan["l"], plan["N"], plan["stride_limbs"], plan["n_fft"]
        L = 1 << l
        X = torch.from_numpy(workloads.residues(w["seed"] + 1000 + k, L, N, stride=st).view(np.int64)).to(device)
        tf, itf = (tg.tft_sqrt2, tg.itft_sqrt2) if plan["sqrt2"] else (tg.tft_ex, tg.itft_ex)

        def three(nn):
            tf(X, l, n, nn, N, 0, st, stream=stream)
            tf(X, l, n, nn, N, 0, st, stream=stream)
            itf(X, l, nn, nn, 0, N, 0, st, scale=1, stream=stream)

        t_trunc = timed(lambda: three(nf))
        t_full = timed(lambda: three(L))
        rows.append([n, l, round(t_mul, 4), round(t_trunc, 4), round(t_full, 4)])
        del F, G, H, X
    mul = [r[2] for r in rows]
    steps = [mul[i + 1] / mul[i] for i in range(len(mul) - 1)]
    return {"workload": f"{len(lengths)} products, equal lengths {lengths[0]} .. {lengths[-1]} in 5 % steps, "
                        f"{bits}-bit unsigned coefficients, ring N = 16384, seed {w['seed']}",
            "columns": ["length", "l", "ms_zx_mul", "ms_3_transforms_truncated", "ms_3_transforms_full_L"],
            "rows": rows,
            "max_step_ratio": round(max(steps), 3),
            "truncated_over_full": round(sum(r[3] for r in rows) / sum(r[4] for r in rows), 4)}


def pointwise_leg(tg, device, stream):
    """Pointwise products mod 2^N + 1 by both methods (schoolbook warp kernel; a second
    Schoenhage-Strassen level on the transform kernels): ms per batch of uniform residues,
    resident in HBM, and whether the two agree bit for bit."""
    import numpy as np
    import torch

    out = {}
    for N, n in ((8192, 20000), (32768, 10000)):
        W = N // 64 + 1
        s = W + (W & 1)
        a = torch.from_numpy(workloads.residues(21, n, N, stride=s).view(np.int64)).to(device)
        b = torch.from_numpy(workloads.residues(22, n, N, stride=s).view(np.int64)).to(device)
        ms, res = {}, {}
        for m in (1, 2):
            x = a.clone()
            tg.pointwise(x, b, n, N, s, m, stream=stream)
            res[m] = x.clone()
            for _ in range(2):
                tg.pointwise(x, b, n, N, s, m, stream=stream)
            torch.cuda.synchronize(device)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                tg.pointwise(x, b, n, N, s, m, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(device)
            ms[m] = e0.elapsed_time(e1) / 5
        plan = tg.pointwise_plan(N, 2)
        out[str(N)] = {"products": n, "ms_schoolbook": round(ms[1], 4), "ms_recursive": round(ms[2], 4),
                       "recursive_k": plan["k"], "inner_N": plan["N_inner"],
                       "auto_method": tg.pointwise_plan(N)["method"], "bit_exact": bool(torch.equal(res[1], res[2]))}
    return out


def run_batch(args):
    import torch

    import paper_0810_3203_gb300 as tg

    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    tg.load()
    res = batch_leg(tg, device, torch.cuda.current_stream(device), args.steps, args.warmup, not args.no_tune)
    print(json.dumps(res), flush=True)
    return 0 if res["bit_exact_vs_plain"] else 1


def run_serve(args):
    import torch

    import paper_0810_3203_gb300 as tg

    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    tg.load()
    res = serve_leg(tg, device, torch.cuda.current_stream(device), args.serve_requests, not args.no_tune,
                    slots=args.serve_slots)
    print(json.dumps(res), flush=True)
    return 0 if res["bit_exact_vs_plain"] else 1


def run_pointwise_case(args):
    """Schoolbook pointwise products a_i <- a_i b_i mod 2^N + 1 at N = 32768 (the case ncu
    captures): 1024 products of 514-limb cells, one warm-up call, then `profile_reps` calls, each
    timed with CUDA events."""
    import numpy as np
    import torch

    import paper_0810_3203_gb300 as tg

    tg.load()
    N, n, s = 32768, 1024, 514
    a = torch.from_numpy(workloads.residues(21, n, N, stride=s).view(np.int64)).cuda()
    b = torch.from_numpy(workloads.residues(22, n, N, stride=s).view(np.int64)).cuda()
    x = a.clone()
    tg.pointwise(x, b, n, N, s, 1)
    ms = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.profile_reps):
        x.copy_(a)
        e0.record()
        tg.pointwise(x, b, n, N, s, 1)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    macs = n * (N // 32) ** 2
    print(json.dumps({"pointwise_case": "1024 products mod 2^32768+1, schoolbook", "ms": [round(v, 4) for v in ms],
                      "mac32_per_s": round(macs / (min(ms) * 1e-3), 1)}))
    return 0


def run_profile_case(args):
    """One TFT and one ITFT at n = 40000 on one 269 MB buffer (the case ncu captures)."""
    import numpy as np
    import torch

    import paper_0810_3203_gb300 as tg

    tg.load()
    N, l, n = WORKLOAD["N"], WORKLOAD["l"], 40000
    if args.config:
        ls_max, ls_c, mw, sp = (int(v) for v in args.config.split(","))
        tg.config_set(N, {"ls_max": ls_max, "ls_c": ls_c, "max_warps": mw, "split": sp})
    if args.fused >= 0:
        tg.config_set(N, dict(tg.config_get(N), fused=args.fused))
    if args.tma >= 0:
        tg.config_set(N, dict(tg.config_get(N), tma=args.tma))
    W = N // 64 + 1
    stride = cell_stride(W, args.stride)
    x = workloads.residues(WORKLOAD["seed"], n, N, stride=stride, cells=1 << l)
    d = torch.from_numpy(x.view(np.int64)).cuda()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_tft, t_itft = [], []
    for _ in range(args.profile_reps):
        ev[0].record()
        tg.tft_ex(d, l, n, n, N, 0, stride)
        ev[1].record()
        tg.itft_ex(d, l, n, n, 0, N, 0, stride, 1)
        ev[2].record()
        ev[2].synchronize()
        t_tft.append(ev[0].elapsed_time(ev[1]))
        t_itft.append(ev[1].elapsed_time(ev[2]))
    torch.cuda.synchronize()
    back = d.view(-1, stride)[:n, :W].cpu().numpy().view(np.uint64)
    ok = bool(np.array_equal(back, x.reshape(-1, stride)[:n, :W]))
    out = {"profile_case": "tft+itft n=40000 l=16 N=32768", "reps": args.profile_reps, "ok": ok,
           "config": tg.config_get(N)}
    if args.profile_reps > 1:  # the first call plans and warms up
        out["tft_ms_median"] = round(float(np.median(t_tft[1:])), 4)
        out["itft_ms_median"] = round(float(np.median(t_itft[1:])), 4)
    print(json.dumps(out))
    return 0 if ok else 1


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", action="store_true",
                    help="run one TFT + ITFT at n = 40000 and exit (the case profiled with ncu)")
    ap.add_argument("--profile-reps", type=int, default=1)
    ap.add_argument("--pointwise-case", action="store_true",
                    help="run only 1024 schoolbook pointwise products at N = 32768 (the case ncu captures)")
    ap.add_argument("--config", default="",
                    help="ls_max,ls_c,max_warps,split: launch configuration for --profile-case")
    ap.add_argument("--stride", type=int, default=0,
                    help="limbs between cells of the large transforms (default: W rounded up to even)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-product batch leg")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch configurations")
    ap.add_argument("--fused", type=int, default=-1,
                    help="launch form of the large transforms (zx_tune_info.fused: 0 one launch per pass, 1 and "
                         "2 persistent, 3 per-pass persistent loops with L2 prefetch, 4 one launch per pass through "
                         "the spill-free kernel); default: the library's")
    ap.add_argument("--tma", type=int, default=-1,
                    help="cell copies of the large transforms (zx_tune_info.tma: 1 one tensor copy per cell, 0 row "
                         "copies and 16-byte stores); default: the library's")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-e1", action="store_true", help="skip the Sec. 5.1-shaped product sweep")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-slots", type=int, default=3, help="stream slots of the serving loop (1 .. 8)")
    ap.add_argument("--serve-only", action="store_true", help="time only the serving leg")
    ap.add_argument("--batch-only", action="store_true",
                    help="time only the 512-product batch against one-at-a-time products")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.pointwise_case:
        return run_pointwise_case(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.batch_only:
        return run_batch(args)
    if args.serve_only:
        return run_serve(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
