#!/usr/bin/env python3
"""Benchmark: MPSM join throughput on one GB300 (or N independent replicas).

One step = one whole join (phases 1-4: sort R runs, splitters + scatter of S,
sort S partitions, search + merge join) of the configured workload, inputs
already resident in HBM.  Metric: (|R| + |S|) / t in M tuples/s (M = 10^6 for
rates; the workload sizes use the paper's M = 2^20).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config NAME] [--impl ours|reference]

Default workload: plain-400M-1600M, |R| = 400*2^20 unique keys (a permutation
of a dense domain), |S| = 1600*2^20 uniform foreign keys, 16-byte tuples.  The
inputs (33.5 GB) are far larger than L2 (129 MB), so every step streams them
from HBM; no flush is needed.

Under torchrun (N > 1) every rank joins its own replica (seed + rank): the
units (tuples) of all ranks over the slowest rank's time give `value`
("scaling": "weak"); the join itself has no cross-GPU exchange.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MPSM join M tuples/s ((|R|+|S|)/t), % HBM roofline; learned+batched vs plain"
UNIT = "M tuples/s"
HOST_TRIES = 3  # e2e host buffers made at most this often until huge pages cover them
MEGA = 1 << 20

# Algorithmic bytes per unit (one read + one write per data-moving phase):
# partitioned side 32 (partition) + 32 (sort) + 16 (join read) per tuple kept,
# run side 32 (sort) + 16 (join read).  Per kernel family: the bytes one launch
# must move at the least for the units it processes.
ALG_BYTES = {
    "scatter_split": ("S tuples", 32),      # read S, write partitioned S (kept tuples)
    "seg_sort": ("tuples sorted", 32),      # read a segment, write it sorted
    "join": ("S' + R tuples", 16),          # read each kept S tuple and each R tuple once
    # fused final sort + join: the work of the S sort pass (32) and of the join's reads (16 per S' and per R
    # tuple); it moves only the reads (16 + 16), so its DRAM traffic sits below these algorithmic bytes
    "sort_join": ("48 B per S' tuple + 16 B per R tuple", None),
    "scatter_radix": ("tuples", 32),        # one radix pass: read + write
    "hist_fine": ("S tuples", 8),           # read the S keys
    "hist_radix": ("tuples", 8),            # read the keys
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="plain-400M-1600M")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=20120145)
    ap.add_argument("--runs", type=int, default=0, help="T_R (0 = automatic)")
    ap.add_argument("--parts", type=int, default=0, help="P, partitions of S (0 = automatic)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-arms", action="store_true", help="skip the learned and batched comparison arms")
    ap.add_argument("--cpu-sample", type=int, default=16, help="CPU baseline runs 1/this of the workload")
    ap.add_argument("--splitter", default="hist", choices=["hist", "learned", "equi-height"])
    ap.add_argument("--fine-bits", type=int, default=0, help="B, fine histogram bits of S (0 = 12)")
    ap.add_argument("--search", default="binary", choices=["binary", "learned", "interp"])
    ap.add_argument("--run-buckets", default="radix", choices=["radix", "learned"],
                    help="bucket function of the runs' first sort pass")
    ap.add_argument("--no-tune", action="store_true", help="batch: skip the autotuner")
    ap.add_argument("--pairs", action="store_true", help="materialise the matching pairs (|S| x 16 B buffer)")
    ap.add_argument("--side", default="s", choices=["s", "r", "smaller"], help="input that is range-partitioned")
    return ap.parse_args()


SPLITTER_MODES = {"hist": 0, "learned": 1, "equi-height": 2}
SEARCH_MODES = {"binary": 0, "learned": 1, "interp": 2}


def _device_array(ptr: int, n: int, dtype):
    """Copy n values of dtype from a device pointer of the plan's view."""
    import numpy as np
    import torch

    nbytes = n * np.dtype(dtype).itemsize

    class _CAI:
        __cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3,
                                    "strides": None}

    return torch.as_tensor(_CAI(), device="cuda").cpu().numpy().view(dtype)


def partition_balance(plan, st):
    """Per partition of the partitioned side: its size n and the run-side tuples r in
    its key range, from the fine histograms and the splitter vector of the last
    join; the largest over the mean of n and of the split-relevant cost
    n log2 n + T n + r (Sec. 4.3), the quantity Fig. 16 balances."""
    import numpy as np

    v = plan.view()
    nb, P, T = int(v.nfine), int(v.partitions_s), int(st["runs_r"])
    if nb == 0 or P == 0:
        return None
    sp = _device_array(v.splitters, nb, np.uint32).astype(np.int64)
    n = np.bincount(sp, weights=_device_array(v.fine_s, nb, np.uint64).astype(np.float64), minlength=P)
    r = np.bincount(sp, weights=_device_array(v.fine_r, nb, np.uint64).astype(np.float64), minlength=P)
    cost = n * np.log2(np.maximum(n, 1.0)) + T * n + r
    return {"parts": P, "fine_buckets": nb, "size_max_over_mean": float(n.max() / n.mean()),
            "cost_max_over_mean": float(cost.max() / cost.mean()),
            "run_side_max_over_mean": float(r.max() / max(r.mean(), 1.0))}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


BATCH_CONFIG = "batch-256"


def workload(name: str, seed: int):
    import gen

    if name not in gen.CONFIGS:
        raise SystemExit(f"unknown config {name}; choose from {sorted(gen.CONFIGS)}")
    return gen.CONFIGS[name](seed)


def sample_workload(w, div: int):
    """The same shape at 1/div of the size (the bounded CPU sample)."""
    import gen

    return gen.Workload(w.kind, max(1, w.n_r // div), max(1, w.n_s // div), w.seed, theta=w.theta,
                        fk_share=w.fk_share)


# ------------------------------------------------------------------ clocks


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _code_only(text: str) -> str:
    """C/CUDA source without comments and with whitespace collapsed: a comment edit
    does not change the kernel, so it must not invalidate a recorded measurement."""
    import re

    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash(files=None, texts=None):
    """Hash of the code (comments dropped) of the CUDA sources a kernel is built from
    (all of csrc when not named); `texts` supplies other versions of the files."""
    d = os.path.join(ROOT, "paper_1207_0145_gb300", "csrc")
    h = hashlib.sha256()
    for fn in sorted(files or os.listdir(d)):
        if texts and fn in texts:
            text = texts[fn]
        else:
            with open(os.path.join(d, fn), encoding="utf-8") as f:
                text = f.read()
        h.update(_code_only(text).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, config: str):
    """DRAM bytes per launch from a committed ncu summary, if its kernel's sources are unchanged."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{config}_traffic.txt")
    try:
        vals = {}
        with open(path) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.strip()
        files = vals.get("sources", "").split() or None
        if vals.get("source_hash") != kernel_source_hash(files):
            return None
        return int(float(vals["dram_bytes_per_launch"]))
    except (OSError, KeyError, ValueError):
        return None


def traffic_per_tuple(config: str):
    """DRAM bytes per (R + S) tuple of one whole join, summed over the kernel families
    of a committed ncu traffic record, if every source file it names is unchanged."""
    path = os.path.join(ROOT, "profiles", f"step_traffic_{config}.txt")
    try:
        vals = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.lstrip().startswith("#"):
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.strip()
        files = vals.get("sources", "").split() or None
        if vals.get("source_hash") != kernel_source_hash(files):
            return None
        return float(vals["dram_bytes_per_tuple"]), vals.get("measured_on", "")
    except (OSError, KeyError, ValueError):
        return None


def host_numa_of(ptr: int, nbytes: int = 1):
    """Pages per NUMA node of the host mappings that overlap [ptr, ptr + nbytes), summed
    (Linux maps and numa_maps), as "N0=pages N1=pages"."""
    try:
        starts = set()
        with open("/proc/self/maps") as f:
            for line in f:
                lo, hi = (int(x, 16) for x in line.split()[0].split("-"))
                if lo < ptr + nbytes and hi > ptr:
                    starts.add(lo)
        nodes = {}
        with open("/proc/self/numa_maps") as f:
            for line in f:
                parts = line.split()
                if int(parts[0], 16) not in starts:
                    continue
                for q in parts[1:]:
                    if q[:1] == "N" and "=" in q:
                        k, v = q.split("=")
                        nodes[k] = nodes.get(k, 0) + int(v)
        return " ".join(f"{k}={v}" for k, v in sorted(nodes.items())) or None
    except (OSError, ValueError):
        return None


def host_huge_bytes_of(ptr: int, nbytes: int = 1):
    """Bytes on transparent huge pages (AnonHugePages) of the host mappings that overlap
    [ptr, ptr + nbytes), summed (Linux smaps), or None."""
    try:
        total, inside = 0, False
        with open("/proc/self/smaps") as f:
            for line in f:
                head = line.split()[0]
                if "-" in head and ":" not in head:
                    lo, hi = (int(x, 16) for x in head.split("-"))
                    inside = lo < ptr + nbytes and hi > ptr
                elif inside and head == "AnonHugePages:":
                    total += int(line.split()[1]) * 1024
        return total
    except (OSError, ValueError):
        return None


def gpu_host_numa(dev: int):
    """The host NUMA node closest to the GPU (cudaDevAttrHostNumaId), or None."""
    import ctypes

    for name in ("libcudart.so", "libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            rt = None
    if rt is None:
        return None
    v = ctypes.c_int(-1)
    return v.value if rt.cudaDeviceGetAttribute(ctypes.byref(v), 134, dev) == 0 else None


def measure_h2d(host, dev, stream, nbytes: int = 4 << 30, reps: int = 3):
    """Host-to-device GB/s of plain copies from the pinned buffer `host` (best of reps)."""
    import torch

    n = min(nbytes, host.numel() * host.element_size())
    src = host.view(torch.uint8).reshape(-1)[:n]
    dst = torch.empty(n, dtype=torch.uint8, device=dev)
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
        e1.synchronize()
        best = max(best, n / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del dst
    return best


def measure_h2d_whole(bufs, dev, stream, chunk: int = 4 << 30):
    """Milliseconds to copy every byte of the pinned buffers `bufs` to the device, in chunks
    of `chunk` bytes into one device buffer (the link over the whole of each buffer, not a
    prefix), and the slowest chunk's GB/s."""
    import torch

    dst = torch.empty(chunk, dtype=torch.uint8, device=dev)
    evs = []
    with torch.cuda.stream(stream):
        for h in bufs:
            src = h.view(torch.uint8).reshape(-1)
            for a in range(0, src.numel(), chunk):
                n = min(chunk, src.numel() - a)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                dst[:n].copy_(src[a:a + n], non_blocking=True)
                e1.record(stream)
                evs.append((n, e0, e1))
    evs[-1][2].synchronize()
    total = sum(e0.elapsed_time(e1) for _, e0, e1 in evs)
    slowest = min(n / (e0.elapsed_time(e1) / 1e3) / 1e9 for n, e0, e1 in evs)
    del dst
    return total, slowest


def cpu_baseline(w, div: int):
    import oracle

    sw = sample_workload(w, div)
    R, S = sw.r_host(), sw.s_host()
    t = time.perf_counter()
    c, k = oracle.join(R, S)
    dt = time.perf_counter() - t
    units = sw.n_r + sw.n_s
    return {"value": units / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"same workload shape at 1/{div}: |R|={sw.n_r}, |S|={sw.n_s} "
                      f"(single-threaded std::sort + merge join, {dt:.1f} s)",
            "seconds": round(dt, 2), "result": [c, k]}


def cpu_pmpsm(w, div: int):
    """The paper's own algorithm, P-MPSM, multithreaded on all host cores (pmpsm_cpu/),
    on the same bounded sample as the oracle baseline: a stronger CPU comparison."""
    import pmpsm_cpu

    sw = sample_workload(w, div)
    R, S = sw.r_host(), sw.s_host()
    cores = os.cpu_count() or 1
    pmpsm_cpu.join(R, S, threads=cores)  # warm-up (page faults of the buffers)
    t = time.perf_counter()
    c, k, ms = pmpsm_cpu.join(R, S, threads=cores)
    dt = time.perf_counter() - t
    return {"value": (sw.n_r + sw.n_s) / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "p-mpsm threads",
            "sample": f"same workload shape at 1/{div}: |R|={sw.n_r}, |S|={sw.n_s}, B = 10, T = {cores}",
            "seconds": round(dt, 3), "phases_ms": [round(x, 1) for x in ms], "result": [c, k]}


def aggregate_replicas(ms_local: float, units_local: int, dist=None, device="cpu"):
    """(ms, M units/s) of N independent replicas: the units of all ranks over the
    slowest rank's time (weak scaling, no data-path collective)."""
    ms, units = ms_local, units_local
    if dist is not None:
        import torch

        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = torch.tensor([units_local], dtype=torch.int64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms, units = float(t.item()), int(u.item())
    return ms, units / (ms / 1e3) / 1e6


# ------------------------------------------------------------------ comparison arms

ARM_WARMUP, ARM_STEPS = 3, 5


def time_joins(plan, R, S, stream, steps: int, warmup: int, local: int):
    """(ms per join, results, clock summary) of `steps` joins after `warmup` untimed ones."""
    import torch

    for _ in range(warmup):
        plan.join(R, S)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [plan.join(R, S) for _ in range(steps)]
        e1.record(stream)
        e1.synchronize()
    return e0.elapsed_time(e1) / steps, res, clk.summary()


def arm_modes(config: str, modes, seed: int, dev, local: int):
    """One workload joined under each of `modes` (label, plan options), the first being
    the plain form; every result checked against the generator's closed form."""
    import torch

    import oracle
    from paper_1207_0145_gb300 import Plan

    w = workload(config, seed)
    units = w.n_r + w.n_s
    expect = {}
    th = threading.Thread(target=lambda: expect.setdefault("v", oracle.closed_form(w)), daemon=True)
    th.start()
    stream = torch.cuda.Stream(device=dev)
    R = torch.empty((w.n_r, 2), dtype=torch.int64, device=dev)
    S = torch.empty((w.n_s, 2), dtype=torch.int64, device=dev)
    with torch.cuda.stream(stream):
        w.fill_r_device(R.data_ptr(), stream.cuda_stream)
        w.fill_s_device(S.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    out = {"workload": config, "n_r": w.n_r, "n_s": w.n_s}
    results = []
    for label, opts in modes:
        plan = Plan(w.n_r, w.n_s, stream=stream.cuda_stream, **opts)
        if label == modes[0][0]:
            th.join()  # the host's expected result is ready before the first timed joins
        ms, res, clk = time_joins(plan, R, S, stream, ARM_STEPS, ARM_WARMUP, local)
        plan.set_flags(timing=True)
        plan.join(R, S)
        st = plan.stats()
        plan.close()
        results += res
        out[label] = {"ms_per_step": ms, "value": units / (ms / 1e3) / 1e6, "unit": UNIT, "steps": ARM_STEPS,
                      "warmup": ARM_WARMUP, "options": opts, "clocks": clk,
                      "imbalance": st["imbalance"], "partitions_s": st["partitions_s"],
                      "levels": [st["levels_r"], st["levels_s"]], "ms_learn": round(st["ms_learn"], 3),
                      "search_probes": st["search_probes"], "part_probes": st["part_probes"],
                      "phases_ms": {k: round(st[k], 3) for k in ("ms_sort_runs", "ms_splitters", "ms_scatter",
                                                                 "ms_sort_partitions", "ms_search", "ms_join")}}
    th.join()
    want = expect.get("v")
    out["parity"] = all(r == want for r in results) if want is not None else None
    out["result"] = list(results[-1])
    a, b = modes[0][0], modes[1][0]
    out["speedup"] = out[a]["ms_per_step"] / out[b]["ms_per_step"]
    out["what"] = f"{b} vs {a} on the same inputs; speedup = ms({a}) / ms({b})"
    del R, S
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ reference arm


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    w = workload(args.config, args.seed)
    div = args.cpu_sample * 2
    sw = sample_workload(w, div)
    R, S = sw.r_host(), sw.s_host()
    for _ in range(args.warmup):
        oracle.join(R, S)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.join(R, S)
        times.append(time.perf_counter() - t)
    units = sw.n_r + sw.n_s
    ms = 1e3 * sum(times) / len(times)
    value = units / (ms / 1e3) / 1e6
    sample = f"same workload shape at 1/{div}: |R|={sw.n_r}, |S|={sw.n_s} per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.config, "n_r": w.n_r, "n_s": w.n_s, "sample_div": div},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm


def run_ours(args):
    import numpy as np
    import torch

    import oracle
    from paper_1207_0145_gb300 import Plan
    from paper_1207_0145_gb300.mpsm import host_tuples

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = workload(args.config, args.seed + rank)
    units = w.n_r + w.n_s

    # expected result from the generator's bookkeeping, on the host, while the GPU warms up
    expect = {}
    th = threading.Thread(target=lambda: expect.setdefault("v", oracle.closed_form(w)), daemon=True)
    th.start()

    stream = torch.cuda.Stream(device=dev)
    R = torch.empty((w.n_r, 2), dtype=torch.int64, device=dev)
    S = torch.empty((w.n_s, 2), dtype=torch.int64, device=dev)
    with torch.cuda.stream(stream):
        w.fill_r_device(R.data_ptr(), stream.cuda_stream)
        w.fill_s_device(S.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    plan = Plan(w.n_r, w.n_s, stream=stream.cuda_stream, runs_r=args.runs, partitions_s=args.parts,
                partition_side={"s": 0, "r": 1, "smaller": 2}[args.side],
                splitter_mode=SPLITTER_MODES[args.splitter], search_mode=SEARCH_MODES[args.search],
                run_buckets={"radix": 0, "learned": 1}[args.run_buckets],
                fine_bits=args.fine_bits)

    # the run side and the partitioned side (swapped under role reversal)
    rev = args.side == "r" or (args.side == "smaller" and w.n_r < w.n_s)
    n_run, n_part = (w.n_s, w.n_r) if rev else (w.n_r, w.n_s)
    pairs = None
    if args.pairs:  # foreign keys: exactly one pair per S tuple
        pairs = torch.empty((w.n_s, 2), dtype=torch.int64, device=dev)
    for _ in range(args.warmup):
        got = plan.join(R, S, pairs)
    st = plan.stats()
    launches_per_step = st["launches"]

    def barrier():
        if dist:
            dist.barrier()

    # ---- device-timed steps
    # the host computes the expected result alongside the warm-up; it must be done
    # before the timed steps, whose launches and pass-count reads need the host cores
    th.join()
    torch.cuda.synchronize()
    barrier()
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        results = []
        for _ in range(args.steps):
            results.append(plan.join(R, S, pairs))
        e1.record(stream)
        e1.synchronize()
    barrier()
    ms, value = aggregate_replicas(e0.elapsed_time(e1) / args.steps, units, dist, dev)

    # ---- per-kernel device time (CUDA events around every launch, separate instrumented steps)
    plan.set_flags(kernel_timing=True)
    kt_steps = min(3, args.steps)
    ktimes = {}
    for _ in range(kt_steps):
        plan.join(R, S, pairs)
        for name, (n, t) in plan.kernel_times().items():
            a = ktimes.setdefault(name, [0, 0.0])
            a[0] += n
            a[1] += t
    plan.set_flags(timing=True)
    plan.join(R, S, pairs)
    st = plan.stats()
    plan.set_flags()
    th.join()
    want = expect.get("v")
    parity = all(r == want for r in results) if want is not None else None

    dom = max(ktimes.items(), key=lambda kv: kv[1][1]) if ktimes else None
    peak, peak_kind = measured_peaks()
    roof = None
    if dom:
        name, (n, t_ms) = dom
        per_launch_ms = t_ms / n
        unit_name, per_unit = ALG_BYTES.get(name, ("tuples", 16))
        if name == "sort_join":
            units_launch = 1
            per_unit = (48 * st["s_kept"] + 16 * n_run) * kt_steps / n
        elif name == "scatter_split":
            units_launch = n_part
        elif name == "join":
            units_launch = (st["s_kept"] + n_run) * kt_steps / n
        elif name == "seg_sort":
            # the runs' final sort; without the fused sort-and-join the partitions' final sort too
            sorted_units = n_run if "sort_join" in ktimes else n_run + st["s_kept"]
            units_launch = sorted_units * kt_steps / n
        else:
            units_launch = (w.n_r + w.n_s) * kt_steps / n
        alg_bytes = per_unit * units_launch
        achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9
        traffic = recorded_traffic(name, args.config)
        roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                "alg_bytes_per_launch": alg_bytes,
                "alg_unit": unit_name if name == "sort_join" else f"{per_unit} B per {unit_name}",
                "ms_per_launch": per_launch_ms}
    alg_step = 80 * st["s_kept"] + 48 * n_run
    roof_step = {"alg_bytes_per_step": alg_step, "achieved": alg_step / (ms / 1e3) / 1e9,
                 "frac": alg_step / (ms / 1e3) / 1e9 / peak}

    # ---- end to end through the host-buffer entry point (pinned memory)
    e2e = None
    if not args.no_e2e and not args.pairs:
        # The host buffers from the library's allocator: page-locked, on transparent huge
        # pages, which the link needs for its full rate.  Right after other processes have
        # released much pinned memory a fresh buffer can get huge pages for only part of its
        # bytes, and one made seconds later all of them: a partly covered buffer is held (so
        # the next one takes other pages) and made again, HOST_TRIES times at most.
        held, host_tries = [], {}

        def huge_host(n, name):
            host_tries[name] = []
            for att in range(HOST_TRIES):
                t = torch.from_numpy(host_tuples(n).view(np.int64))
                cov = host_huge_bytes_of(t.data_ptr(), n * 16)
                host_tries[name].append(cov)
                if not cov or cov >= n * 16 or att == HOST_TRIES - 1:
                    return t
                held.append(t)
                time.sleep(2.0)

        # each buffer filled before the next one is made: the host splits huge pages that
        # hold only zeros when memory runs short, as it does while the next buffer is made
        Rh = huge_host(w.n_r, "R")
        Rh.copy_(R)
        Sh = huge_host(w.n_s, "S")
        Sh.copy_(S)
        held.clear()
        del R, S
        torch.cuda.empty_cache()
        plan.join_host(Rh, Sh)
        torch.cuda.synchronize()
        h2d_before = measure_h2d(Sh, dev, stream)
        # the host link as the timed steps will find it: plain copies of every input byte
        # (on a shared host, parts of a buffer can read at a fraction of the link's rate)
        whole_before, _ = measure_h2d_whole((Rh, Sh), dev, stream)
        barrier()
        fe = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        fe[0].record(stream)
        for i in range(args.steps):
            plan.join_host(Rh, Sh)
            fe[i + 1].record(stream)
        fe[-1].synchronize()
        barrier()
        ems, evalue = aggregate_replicas(fe[0].elapsed_time(fe[-1]) / args.steps, units, dist, dev)
        each = [round(fe[i].elapsed_time(fe[i + 1]), 1) for i in range(args.steps)]
        # the host link as this run saw it, right after the timed steps: plain copies from the
        # same pinned buffers, and where their pages and the GPU sit
        h2d = measure_h2d(Sh, dev, stream)
        whole_ms, whole_min_gbs = measure_h2d_whole((Rh, Sh), dev, stream)
        e2e = {"value": evalue, "unit": UNIT, "h2d_bytes_per_step": units * 16,
               "d2h_bytes_per_step": 16, "ms_per_step": ems,
               "h2d_gbs_measured": round(h2d, 1), "h2d_gbs_before": round(h2d_before, 1),
               "copy_bound_ms": round(units * 16 / (h2d * 1e9) * 1e3, 2),
               "over_copy_bound": round(ems / (units * 16 / (h2d * 1e9) * 1e3), 3),
               "ms_each_step": each, "copy_whole_ms": round(whole_ms, 2),
               "copy_whole_slowest_chunk_gbs": round(whole_min_gbs, 1),
               "copy_whole_ms_before": round(whole_before, 2),
               "over_copy_whole": round(ems / whole_ms, 3),
               "host_alloc": "mpsm_host_alloc (anonymous mapping on transparent huge pages, cudaHostRegister)",
               "host_huge_page_bytes": [host_huge_bytes_of(Rh.data_ptr(), Rh.numel() * 8),
                                        host_huge_bytes_of(Sh.data_ptr(), Sh.numel() * 8)],
               "host_alloc_huge_bytes_per_try": host_tries,
               "host_numa_pinned": host_numa_of(Sh.data_ptr(), Sh.numel() * Sh.element_size()),
               "gpu_host_numa": gpu_host_numa(local),
               "what": "mpsm_join_host: R and S copied from pinned host memory every step, then joined; "
                       "copy_bound_ms = the step's input bytes at the host-to-device rate measured right after the "
                       "timed steps (h2d_gbs_before: the same copy right before them); copy_whole_ms = plain copies of all "
                       "of R and S in 4 GiB chunks, right after (copy_whole_ms_before: right before), and "
                       "over_copy_whole = ms_per_step / copy_whole_ms"}
        del Rh, Sh

    balance = partition_balance(plan, st) if args.splitter != "learned" else None
    plan.close()
    R = S = pairs = None  # noqa: F841 (the device inputs are freed before the comparison arms)
    torch.cuda.empty_cache()
    cpu = cpu_mt = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, args.cpu_sample)
        cpu_mt = cpu_pmpsm(w, args.cpu_sample)
    # the whole step's DRAM traffic from the committed per-kernel ncu record, over the step time
    tr = traffic_per_tuple(args.config)
    hbm_sched = None
    if tr is not None:
        step_bytes = tr[0] * (w.n_r + w.n_s)
        hbm_sched = {"dram_bytes_per_step": step_bytes, "achieved": step_bytes / (ms / 1e3) / 1e9,
                     "peak": peak, "frac": step_bytes / (ms / 1e3) / 1e9 / peak, "unit": "GB/s",
                     "source": f"profiles/step_traffic_{args.config}.txt ({tr[1]})"}
    # learned and batched forms against the plain form (the metric's comparison), default run only
    arms = None
    if ws == 1 and not args.no_arms and args.config == "plain-400M-1600M":
        arms = {
            "zipf": arm_modes("zipf0.9-200M-800M", [("hist", {"splitter_mode": 0}), ("learned", {"splitter_mode": 1})],
                              args.seed, dev, local),
            # learned: the runs' first sort pass and the partitions cut at the sample quantiles of
            # each side; the learned merge-start search alone is timed too
            "sparse": arm_modes("sparse-1600M-1600M", [("binary", {"search_mode": 0}),
                                                       ("learned", {"search_mode": 0, "run_buckets": 1,
                                                                    "splitter_mode": 1}),
                                                       ("learned_search", {"search_mode": 1})],
                                args.seed, dev, local),
        }
        b = batch_measure(args.seed, ARM_STEPS, ARM_WARMUP, True, dev, local)
        arms["batch"] = {"workload": BATCH_CONFIG, "n_r": b["n_r"], "n_s": b["n_s"], "jobs": b["jobs"],
                         "graph": {"ms_per_step": b["ms"], "value": b["value"], "unit": UNIT, "clocks": b["clocks"],
                                   "tuning": b["tuning"], "autotune_ms": b["autotune_ms"]},
                         "sequential": {"ms_per_step": b["seq_ms"], "value": b["seq_value"], "unit": UNIT,
                                        "clocks": b["seq_clocks"]},
                         "parity": b["parity"], "speedup": b["seq_ms"] / b["ms"],
                         "what": "one CUDA-graph launch of all 256 jobs vs 256 mpsm_join calls; "
                                 "speedup = ms(sequential) / ms(graph)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.config, "n_r": w.n_r, "n_s": w.n_s, "tuple_bytes": 16,
                       "runs_r": st["runs_r"], "partitions_s": st["partitions_s"],
                       "l2": "inputs (33.5 GB at the default size) far exceed L2; no flush",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "parity": parity, "result": list(results[-1]),
            "roofline": roof, "roofline_step": roof_step, "hbm_frac_schedule": hbm_sched, "arms": arms,
            "cpu_baseline": cpu, "cpu_pmpsm": cpu_mt, "e2e": e2e, "clocks": clk.summary(),
            "gpu_launches": launches_per_step * args.steps,
            "phases_ms": {k: round(st[k], 3) for k in ("ms_sort_runs", "ms_splitters", "ms_scatter",
                                                       "ms_sort_partitions", "ms_search", "ms_join", "ms_total")},
            "kernels_ms": {k: [v[0], round(v[1] / kt_steps, 3)] for k, v in sorted(ktimes.items(),
                                                                                  key=lambda kv: -kv[1][1])},
            "levels": [st["levels_r"], st["levels_s"]], "imbalance": st["imbalance"],
            "balance": balance,
            "modes": {"splitter": args.splitter, "search": args.search, "run_buckets": args.run_buckets,
                      "pairs": bool(args.pairs),
                      "partitioned": args.side},
            "learned": {k: st[k] for k in ("ms_learn", "loss_s0", "loss_s", "loss_r0", "loss_r", "part_probes",
                                           "search_probes", "search_err", "part_max")},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def batch_measure(seed: int, steps: int, warmup: int, tune: bool, dev, local: int, dist=None):
    """256 independent joins of uneven sizes in one CUDA-graph launch, against the
    same 256 joins run one after another through the single-join entry point."""
    import torch

    import gen
    import oracle
    from paper_1207_0145_gb300 import Plan

    jobs = gen.batch_jobs(256, seed=seed)
    tot_r = sum(j.n_r for j in jobs)
    tot_s = sum(j.n_s for j in jobs)
    units = tot_r + tot_s
    expect = {}
    th = threading.Thread(target=lambda: expect.setdefault("v", [oracle.closed_form(j) for j in jobs]), daemon=True)
    th.start()
    stream = torch.cuda.Stream(device=dev)
    R = torch.empty((tot_r, 2), dtype=torch.int64, device=dev)
    S = torch.empty((tot_s, 2), dtype=torch.int64, device=dev)
    pairs, orr, osr = [], 0, 0
    with torch.cuda.stream(stream):
        for j in jobs:
            r, s_ = R[orr:orr + j.n_r], S[osr:osr + j.n_s]
            j.fill_r_device(r.data_ptr(), stream.cuda_stream)
            j.fill_s_device(s_.data_ptr(), stream.cuda_stream)
            pairs.append((r, s_))
            orr += j.n_r
            osr += j.n_s
    stream.synchronize()
    plan = Plan(tot_r, tot_s, max_jobs=len(jobs), stream=stream.cuda_stream)
    tuning, tune_ms = None, None
    if tune:
        tuning, tune_ms = plan.autotune(pairs, reps=1)
    for _ in range(warmup):
        got = plan.join_batch(pairs)
    th.join()  # the expected results are computed on the host cores before the timed steps
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            got = plan.join_batch(pairs)
        e1.record(stream)
        e1.synchronize()
    if dist:
        dist.barrier()
    ms, value = aggregate_replicas(e0.elapsed_time(e1) / steps, units, dist, dev)
    launches = plan.stats()["launches"]
    # the same jobs one after another through mpsm_join (plain single-join path)
    plan.set_tuning()
    for r, s_ in pairs[:4]:
        plan.join(r, s_)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk2:
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        seq = [plan.join(r, s_) for r, s_ in pairs]
        f1.record(stream)
        f1.synchronize()
    seq_ms = f0.elapsed_time(f1)
    want = expect.get("v")
    res = list(zip(*got))
    parity = (res == want and seq == want) if want is not None else None
    plan.close()
    del R, S, pairs
    torch.cuda.empty_cache()
    return {"ms": ms, "value": value, "units": units, "jobs": len(jobs), "n_r": tot_r, "n_s": tot_s,
            "tuning": tuning, "autotune_ms": tune_ms, "parity": parity, "launches": launches,
            "clocks": clk.summary(), "seq_ms": seq_ms, "seq_value": units / (seq_ms / 1e3) / 1e6,
            "seq_clocks": clk2.summary()}


def run_batch(args):
    import torch

    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    b = batch_measure(args.seed + rank, args.steps, args.warmup, not args.no_tune, dev, local, dist)
    line = {
        "metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": b["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": BATCH_CONFIG, "jobs": b["jobs"], "n_r": b["n_r"], "n_s": b["n_s"], "tuple_bytes": 16,
                   "tuning": b["tuning"], "l2": "inputs far exceed L2; no flush",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "parity": b["parity"], "gpu_launches": b["launches"] * args.steps,
        "sequential": {"value": b["seq_value"], "ms": b["seq_ms"],
                       "what": "the same 256 joins one after another through mpsm_join"},
        "autotune_ms": b["autotune_ms"], "clocks": b["clocks"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == BATCH_CONFIG:
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
