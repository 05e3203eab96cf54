#!/usr/bin/env python
"""ABX benchmark on the triphone-scale synthetic workload.

One step = the whole hot path over one batch: register the 100k items
(features resident in HBM), then for the within-speaker task (on phone, by
context and speaker) and the across-speaker task (on phone, by context,
across speaker): build the cells, compute every needed item-pair distance
(angular frame distances, DTW normalised by path length), score every cell
and collapse (contexts, then speakers, then phone pairs) to an ABX error.

Prints one JSON line.  ``value`` is ABX triplets/s over all ranks with the
features already on the device; ``e2e`` is the same metric through the
public API from pinned host buffers (host->device copy inside the timed
region).  ``--impl reference`` times the FP64 CPU oracle instead, on a
bounded sample of the same workload.

On one GPU the default line also carries ``metric_parts``, the rest of the
metric measured in the same run after the headline: the same step with the
features stored in BF16 and in FP8 E4M3 (interval recheck; flips the FP64
recheck corrected, recheck work, largest distance error on the oracle's
sample, mixed / FP32 throughput), the batched ragged workload in DTW and in
mean-pooled mode, and a short serving run (jobs/s, p50 / p99 job latency).
``--no-extras`` skips them; ``--workload batched`` / ``serve`` give their
full-size lines.
"""
from __future__ import annotations

import argparse
import concurrent.futures
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

from paper_2505_02692_b300 import synth  # noqa: E402

METRIC = "ABX triplets/s & DTW pairs/s on B300, mixed vs FP32; p50/p99 job latency"
TASKS = {
    "within": (synth.PHONE, (synth.CONTEXT, synth.SPEAKER), None),
    "across": (synth.PHONE, (synth.CONTEXT,), synth.SPEAKER),
}
LEVELS = [(synth.CONTEXT,), (synth.SPEAKER,)]
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 148
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) per 128x128 tile of the tile kernels, from one ncu
# capture of the 20k-item across-speaker profiling case (dram__bytes_read.sum
# + dram__bytes_write.sum of the launch / its 22,431 tiles); absent once a
# kernel has changed since it was captured (the BF16 / FP8 instances of the
# narrow kernel have not been captured since its last change).
TRAFFIC_PER_TILE = {"tile_umma_fp32split": (0.769095e9 + 0.707736e9) / 22431}
# DTW kernel, same capture: DRAM bytes per cell ((1.657e9 + 0.122e9) /
# 149,121,283 cells, column-major tiles); the kernel executes about 36
# ALU-pipe thread instructions per cell (sm__inst_executed_pipe_alu.sum x
# thread instructions per instruction / cells = 227,987,313 x 23.57 /
# 149,121,283, counted on an earlier capture of the same loop).
DTW_BYTES_PER_CELL = (1.657254e9 + 0.121915e9) / 149121283
# Algorithmic work of one DP cell: three predecessor compares / minimum, the
# add of the frame distance, the path-length update (about 6 ALU operations),
# and one 4-byte frame distance read.
DTW_ALG_OPS_PER_CELL = 6.0
DTW_ALG_BYTES_PER_CELL = 4.0
ALU_LANES_PER_SM = 64  # 4 schedulers x 16-lane ALU pipe


def dtw_roofline(cells: float, ms: float, peaks: dict) -> dict:
    """Roofline of one DTW launch of `cells` DP cells taking `ms`: algorithmic
    ALU operations (DTW_ALG_OPS_PER_CELL per cell) against the ALU pipe of 148
    SMs x 64 lanes x max SM clock, and algorithmic bytes (one 4-byte distance
    per cell) against the measured HBM bandwidth; the bound is the larger
    fraction."""
    sm_hz = peaks.get("sm_max_mhz", 2032.0) * 1e6
    alu_peak = SM_COUNT * ALU_LANES_PER_SM * sm_hz / 1e12          # Tops/s
    alu_ach = cells * DTW_ALG_OPS_PER_CELL / (ms / 1e3) / 1e12
    hbm_peak = peaks.get("hbm_gbs", 6485.5)
    hbm_ach = cells * DTW_ALG_BYTES_PER_CELL / (ms / 1e3) / 1e9
    r = {"bound": "alu", "unit": "Tops/s", "achieved": alu_ach, "peak": alu_peak,
         "frac": alu_ach / alu_peak, "hbm_achieved_gbs": hbm_ach,
         "hbm_frac": hbm_ach / hbm_peak, "traffic": DTW_BYTES_PER_CELL * cells,
         "traffic_unit": "bytes per launch (ncu DRAM bytes per cell x cells)",
         "peak_source": "derived: 148 SMs x 64 ALU lanes x max SM clock",
         "algorithmic": f"{DTW_ALG_OPS_PER_CELL:.0f} ALU operations and "
                        f"{DTW_ALG_BYTES_PER_CELL:.0f} bytes per DP cell (one per needed "
                        "frame pair)"}
    if r["hbm_frac"] > r["frac"]:
        r.update({"bound": "hbm", "unit": "GB/s", "achieved": hbm_ach, "peak": hbm_peak,
                  "frac": r["hbm_frac"], "peak_source": "measured hbm_gbs",
                  "alu_frac": alu_ach / alu_peak})
    return r


def make_workload(name: str, seed: int):
    if name == "triphone":
        return synth.triphone_scale(seed=seed)
    if name == "tiny":
        return synth.tiny_within(seed=seed)
    # profiling case: 20k items over 40 contexts keeps the triphone workload's
    # 500 items per context (same across-speaker group shape) at 1/5 size
    return synth.make_workload(20000, 768, 40, 40, 40, 3, 25, "skewed", seed,
                               "profile-20k-768")


# Burst GEMM throughput by dtype on a B300 of this machine (TFLOP/s), measured
# with `python bench.py --workload peaks` (cuBLAS through torch, 8192^3):
# MEASURED_PEAKS.json has BF16 only, so the FP8 roofline scales the measured
# BF16 sustained peak by the measured FP8/BF16 ratio.
DTYPE_BURST_TFLOPS = {"bf16": 1765.1, "fp8": 3474.2, "tf32": 965.3, "fp32_simt": 66.0,
                      "fp64": 1.0}
FP8_OVER_BF16 = DTYPE_BURST_TFLOPS["fp8"] / DTYPE_BURST_TFLOPS["bf16"]


def load_peaks():
    try:
        with open(PEAKS_FILE) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
                "sm_max_mhz": 2032.0}, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """SM clock, power and clock-event reasons sampled during a region: NVML
    read-only queries every 10 ms from a thread (nvidia-smi at 200 ms when
    NVML is unavailable).  Nothing is changed on the GPU."""

    REASONS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40),
               ("sw_thermal_slowdown", 0x20), ("sw_power_cap", 0x4),
               ("hw_power_brake", 0x80))
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.nvml = None
        self.samples = []  # (sm_mhz, max_mhz, power_w, reason bits)

    def _handle(self):
        """NVML through ctypes (the driver's libnvidia-ml): read-only queries."""
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        bus = None
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.device)
            bus = b"%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        except Exception:  # noqa: BLE001 -- older torch: use the index
            bus = None
        rc = lib.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(h)) if bus else 1
        if rc != 0 and lib.nvmlDeviceGetHandleByIndex_v2(self.device, ctypes.byref(h)) != 0:
            raise OSError("no NVML handle")
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, h, reasons

    def _poll(self):
        import ctypes
        lib, h, reasons = self.nvml
        sm_clock = 1  # NVML_CLOCK_SM
        v, mx, pw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        lib.nvmlDeviceGetMaxClockInfo(h, sm_clock, ctypes.byref(mx))
        while not self.stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, sm_clock, ctypes.byref(v)) == 0 and
                    reasons(h, ctypes.byref(rs)) == 0):
                p = pw.value / 1e3 if lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(pw)) == 0 else 0.0
                self.samples.append((float(v.value), float(mx.value), p, int(rs.value)))
            self.first.set()
            self.stop.wait(0.01)

    def __enter__(self):
        import threading
        try:
            self.nvml = self._handle()
            self.stop = threading.Event()
            self.first = threading.Event()
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            # the first queries of a process are the slow ones (NVML sets up
            # its device state): let them finish before the timed region
            self.first.wait(2.0)
            return self
        except Exception:  # noqa: BLE001 -- no NVML: nvidia-smi
            self.nvml = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.nvml is not None:
            self.stop.set()
            self.thread.join(timeout=2)
            return False
        if self.proc is None:
            return False
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        bits = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40,
                "sw_thermal_slowdown": 0x20, "sw_power_cap": 0x4}
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != 9 or not parts[1].replace(".", "").isdigit():
                continue
            rs = 0
            for (n, b), v in zip(bits.items(), parts[5:9]):
                if v.lower().startswith("active"):
                    rs |= b
            pw = float(parts[3]) if parts[3].replace(".", "").isdigit() else 0.0
            mx = float(parts[2]) if parts[2].replace(".", "").isdigit() else 0.0
            self.samples.append((float(parts[1]), mx, pw, rs))
        return False

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = sorted({n for _, _, _, rs in self.samples for n, b in self.REASONS if rs & b})
        return {"sm_mhz": statistics.median(s[0] for s in self.samples),
                "sm_max_mhz": max(s[1] for s in self.samples),
                "sm_mhz_min": min(s[0] for s in self.samples),
                "power_w_max": round(max(s[2] for s in self.samples), 1),
                "reasons": reasons, "samples": len(self.samples),
                "source": "nvml 10 ms" if self.nvml is not None else "nvidia-smi 200 ms"}


def clocks_rejected(c) -> bool:
    """A hardware or thermal slowdown, or SM clocks far below max with no
    reason reported (a leftover clock lock), invalidates a measurement."""
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "hw_power_brake"}
    if bad & set(c.get("reasons") or []):
        return True
    sm, mx = c.get("sm_mhz"), c.get("sm_max_mhz")
    return bool(sm and mx and sm < 0.7 * mx and not c.get("reasons"))


# ------------------------------------------------------------- oracle side

def oracle_sample(w, budget_s: float, seed: int = 0, pairs_out=None, mode: str = "dtw"):
    """FP64 oracle on whole contexts of the workload (every within and across
    cell of each chosen context), adding contexts until budget_s of CPU time
    is spent.  Returns (triplets, seconds, contexts, threads).  With pairs_out
    (a dict), the oracle's item-pair distances of each task are added to it as
    pairs_out[task] = list of (x, y, d64) in workload item indices."""
    import oracle
    rng = np.random.default_rng(seed)
    ctxs = rng.permutation(int(w.labels[:, synth.CONTEXT].max()) + 1)
    trip = 0
    secs = 0.0
    used = 0
    for c in ctxs:
        idx = np.flatnonzero(w.labels[:, synth.CONTEXT] == c)
        lens = w.lengths[idx]
        offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        feats = np.concatenate([w.feats[w.offsets[i]:w.offsets[i + 1]] for i in idx])
        labels = w.labels[idx]
        t0 = time.perf_counter()
        for name, (on, by, across) in TASKS.items():
            err, cells, scores, dd = oracle.abx_error(
                feats, offs, labels, on, by, across, LEVELS,
                mode=oracle.MODE_MEAN if mode == "mean" else oracle.MODE_DTW)
            trip += sum(s[1] for s in scores)
            if pairs_out is not None:
                pairs_out.setdefault(name, []).extend(
                    (int(idx[x]), int(idx[y]), v) for (x, y), v in dd.items())
        secs += time.perf_counter() - t0
        used += 1
        if secs >= budget_s:
            break
    return trip, secs, used, oracle.max_threads()


def config_of(args, w, world: int) -> dict:
    """The workload description shared by both arms' JSON lines."""
    lens = w.lengths
    n_lab = [int(w.labels[:, k].max()) + 1 for k in range(3)]
    return {"workload": f"{w.name}: {w.n_items} items, dim {w.dim}, {w.offsets[-1]} frames, "
                        f"lengths {lens.min()}-{lens.max()} (mean {lens.mean():.1f}), "
                        f"{n_lab[0]} phones x {n_lab[1]} contexts x {n_lab[2]} speakers",
            "tasks": "within-speaker (by context, speaker) + across-speaker "
                     "(by context, across speaker), on phone",
            "levels": "context, then speaker, then phone pairs",
            "precision": args.precision, "mode": args.mode,
            "recheck": ["off", "interval", "margin"][args.recheck],
            **({"margin": args.margin} if args.recheck == 2 else {}),
            "l2": ("inputs larger than L2 (features %.2f GB)" if w.feats.nbytes > 126e6 else
                   "inputs fit in L2 (features %.2f GB; not a throughput workload)")
                  % (w.feats.nbytes / 1e9),
            "parallelism": "replicas" if world > 1 else "1 GPU"}


def max_over_ranks(x: float, device: str, dist_on: bool) -> float:
    """The largest x over the ranks of the default process group (the
    slowest rank's time sets a multi-rank step); x itself on one rank."""
    if not dist_on:
        return float(x)
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    w = make_workload(args.workload, 0)
    per_step = []
    trip_total = 0
    t_total = 0.0
    ncontexts = 0
    threads = 1
    for i in range(args.warmup + args.steps):
        trip, secs, used, threads = oracle_sample(w, args.ref_budget, seed=i, mode=args.mode)
        if i >= args.warmup:
            per_step.append(secs)
            trip_total += trip
            t_total += secs
            ncontexts += used
    value = trip_total / t_total
    sample = (f"{ncontexts} context slices of 200 over {args.steps} steps (all within- and "
              f"across-speaker cells of each chosen context), FP64 oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "triplets/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args, w, world),
        "cpu_baseline": {"value": value, "unit": "triplets/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "triplets/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- GPU side

def pipelined_steps(torch, abx, enqueue, finish, feats, steps, stream, step_streams,
                    load_on=None):
    """Run `steps` steps on resident features, enqueueing step k+1 before
    finishing step k.  Step k runs on step_streams[k % len(step_streams)]
    (each stream first waits for `stream`, and `stream` for all of them at
    the end), so that with two streams a step's first kernels can start
    while the previous step's last ones still run.  Returns (triplets,
    pairs)."""
    for sk in step_streams:
        sk.wait_stream(stream)
    trip = pairs = 0
    pend = None
    for k in range(steps):
        with torch.cuda.stream(step_streams[k % len(step_streams)]):
            h = enqueue(feats, abx.MEM_DEVICE_BORROW, load_on=load_on)
        if pend is not None:
            t, p_ = finish(pend)
            trip += t
            pairs += p_
        pend = h
    t, p_ = finish(pend)
    trip += t
    pairs += p_
    for sk in step_streams:
        stream.wait_stream(sk)
    return trip, pairs


def precision_row(abx, torch, ctx, pname, enqueue, finish, d_feats, stats, steps, warmup,
                  sample_pairs, tasks, w, mode, local, step_streams):
    """One more timed run of the headline step (features resident) at another
    storage precision: ms / step, triplets and pairs per second, the FP64
    recheck's work, decision flips it corrected, the top kernels, the DTW
    kernel's roofline, and the largest |d - d64| on the oracle's sample."""
    prec = abx.PRECISIONS[pname]
    for _ in range(warmup):
        finish(enqueue(d_feats, abx.MEM_DEVICE_BORROW))
    torch.cuda.synchronize()
    abx.prof_reset()
    abx.prof_enable(True)
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        trip, pairs = pipelined_steps(torch, abx, enqueue, finish, d_feats, steps, stream,
                                      step_streams)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    prof = abx.prof_read()
    abx.prof_enable(False)
    peaks, _ = load_peaks()
    row = {"ms_per_step": ms / steps, "steps": steps, "warmup": warmup,
           "triplets_per_s": trip / (ms / 1e3), "pairs_per_s": pairs / (ms / 1e3),
           "recheck": "interval (exact)",
           "recheck_pairs": sum(v["recheck_pairs"] for v in stats.values()),
           "recheck_fp64_pairs": sum(v["exact_pairs"] for v in stats.values()),
           "undecided_triples": sum(v["undecided"] for v in stats.values()),
           "flips_before_recheck": sum(v["flips"] for v in stats.values()),
           "errors": {k: v["error"] for k, v in stats.items()},
           "kernels": {k: round(v[0] / steps, 4) for k, v in
                       sorted(prof.items(), key=lambda kv: -kv[1][0])[:6]},
           "clocks": clk.summary()}
    if "dtw" in prof:
        cells = sum(max(v["frame_pairs"], 0) for v in stats.values())
        row["dtw_roofline"] = dtw_roofline(cells, prof["dtw"][0] / steps, peaks)
    if sample_pairs:
        err = 0.0
        items = abx.abx_load_items(ctx, d_feats, w.offsets, w.labels, mem=abx.MEM_DEVICE_BORROW)
        for name, (on, by, across) in tasks.items():
            if name not in sample_pairs:
                continue
            cl = abx.abx_build_cells(ctx, items, on, by, across)
            dd = abx.abx_distances(ctx, items, cl, mode, prec)
            arr = np.array(sample_pairs[name], dtype=np.float64)
            d, _, _, _ = dd.lookup(arr[:, 0].astype(np.int64), arr[:, 1].astype(np.int64))
            err = max(err, float(np.max(np.abs(d - arr[:, 2]))))
            dd.free()
            cl.free()
        items.free()
        row["max_abs_dist_err_sample"] = err
    return row


def run_ours(args, rank: int, world: int):
    import torch
    from paper_2505_02692_b300 import abx

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist_on = world > 1
    if dist_on:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist_on:
            import torch.distributed as tdist
            tdist.barrier()

    w = make_workload(args.workload, rank)
    tasks = TASKS if args.tasks == "both" else {args.tasks: TASKS[args.tasks]}
    prec = abx.PRECISIONS[args.precision]
    mode = abx.MEAN if args.mode == "mean" else abx.DTW
    step_prec = {"prec": prec}  # precision of the steps (the extras re-run others)
    d_feats = torch.from_numpy(w.feats).cuda()
    h_feats = torch.empty(w.feats.shape, dtype=torch.float32, pin_memory=True)
    h_feats.numpy()[:] = w.feats
    ctx = abx.Context(local)
    stream = torch.cuda.current_stream()

    stats = {}
    host = {}

    host_lock = threading.Lock()

    def timed(key, fn, *a, **k):
        t0 = time.perf_counter()
        r = fn(*a, **k)
        with host_lock:
            host[key] = host.get(key, 0.0) + (time.perf_counter() - t0) * 1e3
        return r

    # --plan-threads 2 plans a step's tasks on host threads of their own (the
    # library's calls release the GIL and keep per-thread scratch); measured
    # slower than planning them in turn (19-27 against 15 ms per step: the
    # two threads' allocations, event records and uploads contend), so one
    # thread is the default
    planners = (concurrent.futures.ThreadPoolExecutor(max_workers=len(tasks))
                if args.plan_threads > 1 and len(tasks) > 1 else None)

    def plan_task(items, name, st):
        on, by, across = tasks[name]
        cl = timed("build_cells", abx.abx_build_cells, ctx, items, on, by, across)
        dd = timed("distances", abx.abx_distances, ctx, items, cl, mode, step_prec["prec"],
                   stream=st)
        return cl, dd

    # A step is enqueue + finish.  enqueue loads the items and enqueues every
    # task's work, scoring included, without waiting; finish waits for the
    # scores and frees the step.  The timed loop enqueues step k+1 before it
    # finishes step k, so the host planning of a step (cell tables, pair and
    # tile plans: about 4 ms) runs while the GPU works on the previous one;
    # the items of a step are loaded on a stream of their own so that their
    # uploads do not queue behind the previous step's kernels.
    load_stream = torch.cuda.Stream()
    # the streams the timed steps take in turn (--streams; one: the current)
    step_streams = [stream] + [torch.cuda.Stream() for _ in range(args.streams - 1)]

    def enqueue(feats, mem, items=None, load_on=None):
        if items is None:
            items = timed("load_items", abx.abx_load_items, ctx, feats, w.offsets, w.labels,
                          mem=mem, stream=load_on)
        # across-speaker first when planned in turn: its kernels are the long
        # ones (about 9 of the 13 ms), and the within-speaker planning runs
        # while they do
        order = list(tasks)[::-1]
        st = torch.cuda.current_stream().cuda_stream  # the step's stream, for every thread
        if planners is not None:
            futs = [planners.submit(plan_task, items, name, st) for name in order]
            planned = [f.result() for f in futs]
            cells = {name: r[0] for name, r in zip(order, planned)}
            dists = {name: r[1] for name, r in zip(order, planned)}
        else:
            # every task's cells first: each abx_build_cells waits for its
            # tables from the GPU, and the within-speaker tables, built after
            # the across-speaker distances were enqueued, waited for the
            # across-speaker tile kernel (about 5 ms of host time per step)
            cells = {name: timed("build_cells", abx.abx_build_cells, ctx, items, *tasks[name])
                     for name in order}
            dists = {name: timed("distances", abx.abx_distances, ctx, items, cells[name], mode,
                                 step_prec["prec"], stream=st)
                     for name in order}
        jobs = {name: timed("score", abx.abx_score_submit, ctx, dists[name], cells[name],
                            LEVELS, recheck=args.recheck, margin=args.margin, stream=st)
                for name in order}
        return items, cells, dists, jobs, order

    def finish(h):
        items, cells, dists, jobs, order = h
        trip = pairs = 0
        for name in order:
            err, st = timed("score", jobs[name].wait)
            info = dists[name].info
            trip += st.n_triplets
            pairs += info.n_pairs
            stats[name] = {"error": err, "triplets": st.n_triplets, "cells": st.n_cells,
                           "pairs": info.n_pairs, "tiles": info.n_tiles,
                           "frame_pairs": info.n_frame_pairs,
                           "undecided": st.n_undecided, "recheck_pairs": st.n_recheck_pairs,
                           "exact_pairs": st.n_exact_pairs, "flips": st.n_flips}
        for name in order:
            dists[name].free()
            cells[name].free()
        items.free()
        return trip, pairs

    def step(feats, mem, items=None):
        return finish(enqueue(feats, mem, items))

    for _ in range(args.warmup):
        step(d_feats, abx.MEM_DEVICE_BORROW)
    torch.cuda.synchronize()
    host.clear()

    # ---- timed region, features resident in HBM; taken once more if the
    # clocks show a slowdown (or sit far below max with no reason given)
    for attempt in range(2):
        host.clear()
        abx.prof_reset()
        abx.prof_enable(True)
        l0 = abx.kernel_launches()
        barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            ev0.record(stream)
            load_stream.wait_stream(stream)
            trip, pairs = pipelined_steps(torch, abx, enqueue, finish, d_feats, args.steps,
                                          stream, step_streams, load_stream.cuda_stream)
            stream.wait_stream(load_stream)
            ev1.record(stream)
            torch.cuda.synchronize()
        barrier()
        if not clocks_rejected(clk.summary()):
            break
    remeasured = attempt > 0
    launches = abx.kernel_launches() - l0
    host_ms = {k: v / args.steps for k, v in host.items()}
    prof = abx.prof_read()
    abx.prof_enable(False)
    ms_max = max_over_ranks(ev0.elapsed_time(ev1), "cuda", dist_on)
    trip_per_step = trip // args.steps
    pairs_per_step = pairs // args.steps
    value = trip_per_step * args.steps * world / (ms_max / 1e3)
    pairs_s = pairs_per_step * args.steps * world / (ms_max / 1e3)

    # ---- end to end: pinned host features through the public API
    # Each step's features are copied from pinned host memory on a second
    # stream while the previous step's kernels run (double buffering): the
    # copy of step k+1 is enqueued before step k's work.  The kernels run on
    # a stream of their own too, since the legacy default stream would wait
    # for the copy stream.
    e2e = None
    if not args.no_e2e:
        copy = torch.cuda.Stream()
        comp = torch.cuda.Stream()

        def load_host():
            return abx.abx_load_items(ctx, h_feats.numpy(), w.offsets, w.labels,
                                      mem=abx.MEM_HOST, stream=copy.cuda_stream)

        torch.cuda.synchronize()
        with torch.cuda.stream(comp):
            step(None, None, items=load_host())
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(comp)
            nxt = load_host()
            for k in range(args.steps):
                cur = nxt
                if k + 1 < args.steps:
                    nxt = load_host()
                step(None, None, items=cur)
            e1.record(comp)
            torch.cuda.synchronize()
        ems = e0.elapsed_time(e1)
        wall = (time.perf_counter() - t0) * 1e3
        emax = max_over_ranks(max(ems, wall), "cuda", dist_on)
        h2d = w.feats.nbytes + w.offsets.nbytes + w.labels.nbytes
        d2h = 2 * (8 + 7 * 8)  # error + stats of both tasks
        e2e = {"value": trip_per_step * args.steps * world / (emax / 1e3), "unit": "triplets/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h,
               "ms_per_step": emax / args.steps,
               "overlap": "each step's host-to-device copy runs on a second stream during the "
                          "previous step's kernels"}

    if rank != 0:
        if dist_on:
            import torch.distributed as tdist
            tdist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (live CUDA-event times)
    peaks, peak_src = load_peaks()
    top = max(prof.items(), key=lambda kv: kv[1][0]) if prof else ("none", (0.0, 0))
    name, (kms, kn) = top
    fp_step = sum(max(s["frame_pairs"], 0) for s in stats.values())
    tiles_step = sum(s["tiles"] for s in stats.values())
    dim = w.dim
    per_tile = TRAFFIC_PER_TILE.get(name)
    traffic = per_tile * tiles_step * args.steps / kn if (per_tile and kn) else None
    roof = {"kernel": name, "launches": kn, "ms_total": kms, "traffic": traffic,
            "traffic_unit": "bytes per launch (ncu per-tile DRAM bytes x tiles)"}
    if name.startswith("tile"):
        flops = 2.0 * dim * fp_step * args.steps
        achieved = flops / (kms / 1e3) / 1e12
        if name == "tile_simt":
            peak = SM_COUNT * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
            roof.update({"bound": "alu", "unit": "TFLOP/s",
                         "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 x max SM clock"})
        else:
            peak = peaks["bf16_tflops_sustained"]
            src = f"{peak_src} bf16_tflops_sustained"
            if args.precision == "fp8":
                peak *= FP8_OVER_BF16
                src += f" x {FP8_OVER_BF16:.3f} (measured fp8/bf16 cuBLAS ratio)"
            roof.update({"bound": "tensor", "unit": "TFLOP/s", "peak_source": src})
            if args.precision == "fp32":
                roof["note"] = ("FP32 products run as 3 FP16 MMAs (hi*hi + hi*lo + lo*hi), and "
                                "whole 128x128 tiles are computed, so the algorithmic rate "
                                "is at most peak/3 x the needed share of each tile")
            # the MMA work the kernel issues: every 128 x 128 tile of the plan
            # over the padded dimension, 3 FP16 passes for the FP32 split (an
            # upper bound: tiles without a needed pair are skipped)
            passes = 3 if args.precision == "fp32" else 1
            dim_pad = (dim + 127) // 128 * 128
            issued = passes * 2.0 * dim_pad * 128 * 128 * tiles_step * args.steps
            roof["issued_tflops"] = issued / (kms / 1e3) / 1e12
            roof["issued_frac_of_burst"] = roof["issued_tflops"] / (
                peaks.get("bf16_tflops", 1765.0) * (FP8_OVER_BF16 if args.precision == "fp8"
                                                   else 1.0))
        roof.update({"achieved": achieved, "peak": peak, "frac": achieved / peak,
                     "algorithmic": "2 * dim * sum over needed pairs of Tx*Ty"})
    elif name == "dtw":
        roof.update(dtw_roofline(fp_step * args.steps / kn, kms / kn, peaks))
    else:
        roof.update({"bound": "unknown", "achieved": None, "peak": None, "frac": None})
    kernels = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}

    cpu = None
    agree = None
    agree_pairs = None
    if not args.no_cpu_baseline and rank == 0:
        sampled = {}
        trip_s, secs, used, threads = oracle_sample(w, args.ref_budget, pairs_out=sampled,
                                                    mode=args.mode)
        cpu = {"value": trip_s / secs, "unit": "triplets/s", "cores": threads, "kind": "oracle",
               "sample": f"{used} of 200 context slices (all within- and across-speaker "
                         f"cells of each), {secs:.1f} s FP64 oracle"}
        # the same sample's pair distances against one more (untimed) GPU run
        agree = {"pairs": 0, "max_abs_dist_err": 0.0}
        agree_pairs = sampled
        items = abx.abx_load_items(ctx, d_feats, w.offsets, w.labels, mem=abx.MEM_DEVICE_BORROW)
        for name, (on, by, across) in tasks.items():
            if name not in sampled:
                continue
            cl = abx.abx_build_cells(ctx, items, on, by, across)
            dd = abx.abx_distances(ctx, items, cl, mode, prec)
            arr = np.array(sampled[name], dtype=np.float64)
            d, _, _, _ = dd.lookup(arr[:, 0].astype(np.int64), arr[:, 1].astype(np.int64))
            agree["pairs"] += len(arr)
            agree["max_abs_dist_err"] = max(agree["max_abs_dist_err"],
                                            float(np.max(np.abs(d - arr[:, 2]))))
            dd.free()
            cl.free()
        items.free()
        if args.recheck == 2:
            agree["margin"] = args.margin
            agree["margin_covers_sample"] = bool(2 * agree["max_abs_dist_err"] < args.margin)

    # ---- the rest of the metric, on one GPU: the same workload stored in
    # BF16 and FP8 (interval recheck), the batched workload (DTW and mean
    # pooling) and a short serving run
    parts = None
    head_stats = {k: dict(v) for k, v in stats.items()}  # the extras' steps overwrite stats
    if not args.no_extras and world == 1 and args.workload == "triphone":
        parts = {"note": "each part measured in this run after the headline; see the "
                         "--workload batched / serve lines for the full-size versions"}
        rows = {}
        sample_pairs = agree_pairs if agree is not None else None
        for pname in ("bf16", "fp8"):
            step_prec["prec"] = abx.PRECISIONS[pname]
            rows[pname] = precision_row(abx, torch, ctx, pname, enqueue, finish, d_feats,
                                        stats, min(args.steps, 5), 2, sample_pairs, tasks,
                                        w, mode, local, step_streams)
        step_prec["prec"] = prec
        rows[args.precision] = {"ms_per_step": ms_max / args.steps, "triplets_per_s": value,
                                "pairs_per_s": pairs_s,
                                "recheck_pairs": sum(v["recheck_pairs"]
                                                     for v in head_stats.values()),
                                "flips_before_recheck": sum(v["flips"]
                                                            for v in head_stats.values()),
                                "max_abs_dist_err_sample": (agree or {}).get(
                                    "max_abs_dist_err")}
        parts["precision"] = rows
        parts["mixed_vs_fp32"] = {p_: rows[p_]["triplets_per_s"] / value
                                  for p_ in ("bf16", "fp8")}
        del d_feats
        torch.cuda.empty_cache()
        for bmode in ("dtw", "mean"):
            a2 = argparse.Namespace(**{**vars(args), "workload": "batched", "steps": 3,
                                       "warmup": 2, "mode": bmode, "no_cpu_baseline": True})
            bl = run_batched(a2, rank, world)
            parts[f"batched_{bmode}"] = {k: bl[k] for k in ("value", "unit", "ms_per_step",
                                                           "pairs_per_s", "create_s")}
            parts[f"batched_{bmode}"]["roofline_frac"] = (bl["roofline"] or {}).get("frac")
            parts[f"batched_{bmode}"]["workload"] = bl["config"]["workload"]
        a3 = argparse.Namespace(**{**vars(args), "workload": "serve", "jobs": 120, "warmup": 3,
                                   "no_cpu_baseline": True, "precision": "bf16"})
        sl = run_serve(a3, rank, world)
        parts["serving"] = {"jobs": 120, "jobs_per_s": sl["value"], "p50_ms": sl["p50_ms"],
                            "p99_ms": sl["p99_ms"], "solo_p50_ms": sl["solo_p50_ms"],
                            "solo_p99_ms": sl["solo_p99_ms"],
                            "mean_jobs_per_batch": sl["loads"]["0.8"]["mean_jobs_per_batch"],
                            "load": "Poisson at 0.8x the solo job rate (0.5x in loads)",
                            "loads": sl["loads"]}

    line = {
        "metric": METRIC, "value": value, "unit": "triplets/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32_simt": "f32", "fp32": "f32 (fp16x3 split products, f32 accumulate)",
                  "bf16": "bf16 storage, f32 accumulate", "fp8": "e4m3 storage, f32 accumulate"}
        [args.precision],
        "data": "synthetic",
        "config": {**config_of(args, w, world),
                   "pipelining": "step k+1 is planned and enqueued before step k's scores "
                                 "are read; all K steps complete inside the timed region",
                   "planning": f"{args.plan_threads} host thread(s) plan a step's tasks"},
        "pairs_per_s": pairs_s,
        "per_task": head_stats,
        "roofline": roof,
        "kernels": kernels,
        "kernels_note": "CUDA-event time per launch on its stream; the cell-building, scan "
                        "and upload kernels run on side streams while the previous step's "
                        "kernels occupy the SMs, so their times include waiting for an SM",
        "host_ms_per_step": host_ms,
        "cpu_baseline": cpu,
        "vs_oracle_sample": agree,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": dict(clk.summary(), remeasured=remeasured),
        "metric_parts": parts,
    }
    print(json.dumps(line), flush=True)
    if dist_on:
        import torch.distributed as tdist
        tdist.destroy_process_group()


# ------------------------------------------------------- batched tasks

def batched_oracle_sample(specs, tasks, budget_s: float, mode: str):
    """FP64 oracle on whole tasks of the batch, smallest first, until budget_s
    of CPU time is spent.  Returns (triplets, seconds, tasks used, threads,
    {task index: oracle error})."""
    import oracle
    order = sorted(range(len(specs)), key=lambda k: specs[k].n_items)
    trip, secs, errs = 0, 0.0, {}
    on, by, across = TASKS["within"]
    for k in order:
        feats, offs, labels = tasks[k]
        f = feats.cpu().numpy() if hasattr(feats, "cpu") else feats
        t0 = time.perf_counter()
        err, cells, scores, _ = oracle.abx_error(
            f, offs, labels, on, by, across, LEVELS,
            mode=oracle.MODE_MEAN if mode == "mean" else oracle.MODE_DTW)
        secs += time.perf_counter() - t0
        trip += sum(sc[1] for sc in scores)
        errs[k] = err
        if secs >= budget_s:
            break
    return trip, secs, len(errs), oracle.max_threads(), errs


def run_batched(args, rank: int, world: int):
    """Batched ragged tasks: 64 independent within-speaker tasks of mixed
    dimensions in shared launches, one CUDA-graph replay per step."""
    import torch
    from paper_2505_02692_b300 import abx

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    specs = synth.batched_specs(seed=rank)
    tasks = [synth.make_task_device(sp, device=f"cuda:{local}") for sp in specs]
    ctx = abx.Context(local)
    prec = abx.PRECISIONS[args.precision]
    mode = abx.MEAN if args.mode == "mean" else abx.DTW
    on, by, across = TASKS["within"]
    t0 = time.perf_counter()
    b = abx.abx_batch_create(ctx, tasks, on, by, across, mode, prec, LEVELS,
                             recheck=args.recheck, margin=args.margin, tune=True)
    create_s = time.perf_counter() - t0
    feat_bytes = sum(t[0].numel() * 4 for t in tasks)
    host_tasks = None
    if not args.no_cpu_baseline and rank == 0:
        # keep the small tasks' features on the host for the oracle sample
        order = sorted(range(len(specs)), key=lambda k: specs[k].n_items)[:8]
        host_tasks = {k: (tasks[k][0].cpu().numpy(), tasks[k][1], tasks[k][2]) for k in order}
    del tasks
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        b.run()
    err, trip, st = b.wait()
    info = b.info
    torch.cuda.synchronize()
    l0 = abx.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            b.run()
        ev1.record(stream)
        err, trip, st = b.wait()
    launches = abx.kernel_launches() - l0
    ms = ev0.elapsed_time(ev1)
    info = b.info
    n_trip = int(trip.sum())
    value = n_trip * args.steps / (ms / 1e3)
    # one eager run with per-kernel events for the roofline
    b.set_graph(False)
    abx.prof_reset()
    abx.prof_enable(True)
    b.run()
    b.wait()
    prof = abx.prof_read()
    abx.prof_enable(False)
    b.set_graph(True)
    peaks, peak_src = load_peaks()
    tile = {k: v for k, v in prof.items() if k.startswith("tile")}
    roof = None
    if tile and mode == abx.DTW:
        kms = sum(v[0] for v in tile.values())
        name = max(tile, key=lambda k: tile[k][0])
        peak = peaks["bf16_tflops_sustained"] * (FP8_OVER_BF16 if args.precision == "fp8" else 1.0)
        ach = info.flops / (kms / 1e3) / 1e12
        roof = {"kernel": name, "launches": sum(v[1] for v in tile.values()), "ms_total": kms,
                "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None,
                "peak_source": f"{peak_src} bf16_tflops_sustained",
                "algorithmic": "sum over classes of 2 * dim * needed frame pairs"}
    kernels = {k: {"ms_per_run": v[0], "launches_per_run": v[1]}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}
    cpu = None
    if host_tasks is not None:
        hs = [host_tasks.get(k) for k in range(len(specs))]
        trip_s, secs, used, threads, errs = batched_oracle_sample(
            [specs[k] for k in host_tasks], [host_tasks[k] for k in host_tasks],
            args.ref_budget, args.mode)
        keys = list(host_tasks)
        agree = all(err[keys[i]] == e for i, e in errs.items())
        cpu = {"value": trip_s / secs, "unit": "triplets/s", "cores": threads, "kind": "oracle",
               "sample": f"{used} smallest of {len(specs)} tasks (all cells), {secs:.1f} s "
                         "FP64 oracle", "errors_identical": bool(agree)}
        del hs
    dims = sorted({sp.dim for sp in specs})
    line = {
        "metric": METRIC, "value": value, "unit": "triplets/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32_simt": "f32", "fp32": "f32 (fp16x3 split products, f32 accumulate)",
                  "bf16": "bf16 storage, f32 accumulate", "fp8": "e4m3 storage, f32 accumulate"}
        [args.precision],
        "data": "synthetic",
        "config": {"workload": f"batched: {len(specs)} tasks, {sum(sp.n_items for sp in specs)} "
                               f"items (1k-50k log-uniform), dims {dims}, lengths 3-40 skewed "
                               "short, 10-60 phones, 20 contexts x 4 speakers",
                   "tasks": "within-speaker (by context, speaker), on phone",
                   "levels": "context, then speaker, then phone pairs",
                   "precision": args.precision, "mode": args.mode,
                   "recheck": ["off", "interval", "margin"][args.recheck],
                   "launch": f"one CUDA graph per step ({info.graph_kernels} kernel nodes, "
                             f"{info.n_classes} dimension classes)",
                   "l2": "inputs larger than L2 (features %.1f GB)" % (feat_bytes / 1e9),
                   "parallelism": "1 GPU"},
        "pairs_per_s": info.n_pairs * args.steps / (ms / 1e3),
        "triplets_per_step": n_trip, "pairs_per_step": info.n_pairs,
        "frame_pairs_per_step": info.n_frame_pairs,
        "tuned": {"class_dim": list(info.class_dim)[:info.n_classes],
                  "tile_variant": list(info.tile_variant)[:info.n_classes],
                  "dtw_variant": list(info.dtw_variant)[:info.n_classes]},
        "create_s": create_s,
        "roofline": roof, "kernels_eager_run": kernels,
        "cpu_baseline": cpu, "e2e": None,
        "gpu_launches": launches, "clocks": clk.summary(),
        "stats": {"undecided": st.n_undecided, "recheck_pairs": st.n_recheck_pairs,
                  "recheck_fp64_pairs": st.n_exact_pairs, "flips": st.n_flips},
    }
    b.free()
    return line


# ------------------------------------------------------------- serving

def run_serve(args, rank: int, world: int):
    """Serving loop: 500 jobs (42 dumps x 12 layers, last dump partial) with
    Poisson arrivals at 0.8x and 0.5x the measured solo job rate; BF16 with
    the recheck; within- and across-speaker specs; admission by free HBM."""
    import torch
    from paper_2505_02692_b300 import abx

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    n_jobs, layers = args.jobs, 12
    dumps = synth.served_dumps(seed=rank, n_dumps=(n_jobs + layers - 1) // layers)
    jobs = [(d, l) for d in range(len(dumps)) for l in range(layers)][:n_jobs]
    prec = abx.PRECISIONS["bf16" if args.precision == "fp32" else args.precision]
    specs = [abx.task_spec(*TASKS[t], LEVELS) for t in ("within", "across")]

    def make(k):
        d, l = jobs[k]
        return synth.make_task_device(dumps[d], device=dev, feat_seed=dumps[d].seed * 100 + l)

    def serve(srv, arrivals):
        """Submit job k at arrivals[k] (seconds from start); collect results."""
        pending, results = {}, {}
        t0 = srv.now()
        k = 0
        nxt = make(0)
        while k < n_jobs or pending:
            while k < n_jobs and srv.now() - t0 >= arrivals[k]:
                pending[srv.submit(*nxt)] = (k, nxt)
                k += 1
                nxt = make(k) if k < n_jobs else None
            for t in list(pending):
                r = srv.poll(t)
                if r is not None:
                    results[pending.pop(t)[0]] = r
            time.sleep(0.0002)
        return results

    ctx = abx.Context(local)
    # warm-up and autotune on a few jobs, then the solo rate: one job at a time
    srv = abx.Server(ctx, 3, specs, abx.DTW, prec, recheck=args.recheck, margin=args.margin,
                     max_inflight=args.serve_executors, max_batch_jobs=32, tune=True,
                     n_planners=args.serve_planners)
    # warm-up: the first job of every feature dimension (the autotuner times
    # its kernel variants once per dimension and keeps the choice), then
    # args.warmup more
    first_of_dim = {}
    for k, (d, _) in enumerate(jobs):
        first_of_dim.setdefault(dumps[d].dim, k)
    for k in list(first_of_dim.values()) + list(range(min(args.warmup, n_jobs))):
        srv.wait(srv.submit(*make(k)))
    rng = np.random.default_rng(1234 + rank)
    solo_idx = sorted(rng.choice(n_jobs, size=min(40, n_jobs), replace=False))
    solo = []
    for k in solo_idx:
        r = srv.wait(srv.submit(*make(k)))
        solo.append(r.t_done - r.t_submit)
    solo_rate = 1.0 / float(np.mean(solo))
    # the solo latencies' own spread (job sizes span 2k-100k items, dims
    # 512-1280): the floor under any p99 / p50 ratio under load
    solo_p50, solo_p99 = (1e3 * float(np.percentile(solo, q)) for q in (50, 99))
    out = {}
    for load in (0.8, 0.5):
        lam = load * solo_rate
        gaps = rng.exponential(1.0 / lam, size=n_jobs)
        arrivals = np.cumsum(gaps) - gaps[0]
        l0 = abx.kernel_launches()
        st0 = srv.stats
        with ClockSampler(local) as clk:
            res = serve(srv, arrivals)
        st1 = srv.stats
        lat = np.array([res[k].t_done - res[k].t_submit for k in range(n_jobs)])
        wait_q = np.array([res[k].t_admit - res[k].t_submit for k in range(n_jobs)])
        plan_w = np.array([res[k].t_launch - res[k].t_admit for k in range(n_jobs)])
        run_t = np.array([res[k].t_done - res[k].t_launch for k in range(n_jobs)])
        t_first = min(res[k].t_submit for k in res)
        t_last = max(res[k].t_done for k in res)
        trip = sum(int(res[k].triplets[0] + res[k].triplets[1]) for k in res)
        failed = sum(1 for k in res if res[k].status != 0)
        out[load] = {"lambda_jobs_per_s": lam, "jobs_per_s": n_jobs / (t_last - t_first),
                     "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                     "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                     "mean_ms": 1e3 * float(lat.mean()),
                     "p50_parts_ms": {"queued": 1e3 * float(np.median(wait_q)),
                                      "planned_and_waiting": 1e3 * float(np.median(plan_w)),
                                      "on_gpu": 1e3 * float(np.median(run_t))},
                     "triplets_per_s": trip / (t_last - t_first),
                     "batches": st1.batches - st0.batches,
                     "mean_jobs_per_batch": n_jobs / max(1, st1.batches - st0.batches),
                     "max_inflight": st1.max_inflight_seen, "failed": failed,
                     "peak_gb": st1.peak_bytes / 1e9,
                     "gpu_launches": abx.kernel_launches() - l0, "clocks": clk.summary()}
    srv.close()
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        import oracle
        small = sorted(range(len(dumps)), key=lambda d: dumps[d].n_items)[:2]
        trip_s, secs = 0, 0.0
        used = 0
        for d in small:
            f, o, lab = synth.make_task_device(dumps[d], device=dev, feat_seed=dumps[d].seed * 100)
            f = f.cpu().numpy()
            t0 = time.perf_counter()
            for t in ("within", "across"):
                on, by, across = TASKS[t]
                _, _, scores, _ = oracle.abx_error(f, o, lab, on, by, across, LEVELS)
                trip_s += sum(sc[1] for sc in scores)
            secs += time.perf_counter() - t0
            used += 1
            if secs >= args.ref_budget:
                break
        cpu = {"value": trip_s / secs, "unit": "triplets/s", "cores": oracle.max_threads(),
               "kind": "oracle", "sample": f"{used} smallest dumps (layer 0, both tasks, all "
                                           f"cells), {secs:.1f} s FP64 oracle"}
    main_load = out[0.8]
    line = {
        "metric": METRIC, "value": main_load["jobs_per_s"], "unit": "jobs/s",
        "n_gpus": world, "steps": n_jobs, "warmup": args.warmup,
        "ms_per_step": main_load["mean_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {abx.BF16: "bf16 storage, f32 accumulate", abx.FP8: "e4m3 storage, f32 accumulate",
                  abx.FP32: "f32 (fp16x3 split products, f32 accumulate)",
                  abx.FP32_SIMT: "f32"}[prec],
        "data": "synthetic",
        "config": {"workload": f"serving: {n_jobs} jobs = {len(dumps)} dumps x {layers} layers "
                               "(last partial), items 2k-100k log-uniform, dims "
                               "{512,768,1024,1280}, lengths 3-25 skewed short, 40 phones x "
                               "200 contexts x 40 speakers",
                   "tasks": "within- and across-speaker per job",
                   "arrivals": "Poisson at 0.8x (headline) and 0.5x the solo job rate",
                   "admission": f"FIFO, device-memory budget (80% of free HBM), up to 32 jobs "
                                f"per batch; {args.serve_planners} planner thread(s) batching just "
                                f"in time, {args.serve_executors} executor(s) with a stream each",
                   "recheck": ["off", "interval", "margin"][args.recheck],
                   "parallelism": "1 GPU"},
        "p50_ms": main_load["p50_ms"], "p99_ms": main_load["p99_ms"],
        "solo_jobs_per_s": solo_rate, "solo_mean_ms": 1e3 * float(np.mean(solo)),
        "solo_p50_ms": solo_p50, "solo_p99_ms": solo_p99,
        "loads": {str(k): v for k, v in out.items()},
        "cpu_baseline": cpu, "e2e": None,
        "gpu_launches": main_load["gpu_launches"], "clocks": main_load["clocks"],
    }
    return line


def run_peaks(args, rank: int, world: int):
    """Library throughput of the dtypes the roofline lines need and
    MEASURED_PEAKS.json lacks: TF32, FP8 E4M3 (cuBLASLt, BF16 out), FP32 on
    the CUDA cores and FP64 GEMMs (2 n^3 FLOP, best of several, CUDA events),
    plus the BF16 GEMM and an HBM copy for comparison.  Prints one JSON line."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"

    def best_ms(fn, reps=10):
        fn()
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    out = {}
    with ClockSampler(local) as clk:
        n = 8192
        a = torch.randn(n, n, device=dev, dtype=torch.bfloat16)
        b = torch.randn(n, n, device=dev, dtype=torch.bfloat16)
        out["bf16_tflops"] = 2 * n ** 3 / best_ms(lambda: a @ b) / 1e9
        a32, b32 = a.float(), b.float()
        torch.backends.cuda.matmul.allow_tf32 = True
        out["tf32_tflops"] = 2 * n ** 3 / best_ms(lambda: a32 @ b32) / 1e9
        torch.backends.cuda.matmul.allow_tf32 = False
        out["fp32_simt_tflops"] = 2 * n ** 3 / best_ms(lambda: a32 @ b32, 3) / 1e9
        try:
            a8 = a.to(torch.float8_e4m3fn)
            b8 = b.t().contiguous().to(torch.float8_e4m3fn).t()
            one = torch.ones((), device=dev)
            out["fp8_tflops"] = 2 * n ** 3 / best_ms(
                lambda: torch._scaled_mm(a8, b8, one, one, out_dtype=torch.bfloat16)) / 1e9
        except Exception as e:  # noqa: BLE001 -- report why
            out["fp8_tflops"] = None
            out["fp8_error"] = str(e).splitlines()[0][:200]
        del a, b, a32, b32
        m = 4096
        a64 = torch.randn(m, m, device=dev, dtype=torch.float64)
        out["fp64_tflops"] = 2 * m ** 3 / best_ms(lambda: a64 @ a64, 3) / 1e9
        del a64
        x = torch.empty(1 << 30, device=dev, dtype=torch.bfloat16)
        y = torch.empty_like(x)
        out["hbm_gbs"] = 2 * x.numel() * 2 / best_ms(lambda: y.copy_(x)) / 1e6
    out = {k: (round(v, 1) if isinstance(v, float) else v) for k, v in out.items()}
    if rank == 0:
        print(json.dumps({"workload": "peaks", "burst": out, "clocks": clk.summary(),
                          "how": "torch/cuBLAS GEMMs 8192^3 (FP64 4096^3), best of repeats, "
                                 "CUDA events; copy of 1 Gi bf16 elements (read + write)"}))


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32_simt", "fp32", "bf16", "fp8"],
                    default="fp32")
    ap.add_argument("--mode", choices=["dtw", "mean"], default="dtw")
    ap.add_argument("--recheck", type=int, default=1,
                    help="0 off, 1 FP64 recheck of overlapping intervals (exact), "
                         "2 FP64 recheck of triples whose margin is below --margin")
    ap.add_argument("--margin", type=float, default=0.0)
    ap.add_argument("--workload", choices=["triphone", "tiny", "profile", "batched", "serve",
                                           "peaks"],
                    default="triphone")
    ap.add_argument("--jobs", type=int, default=500, help="jobs of the serving workload")
    ap.add_argument("--serve-executors", type=int, default=1,
                    help="serving: executor threads (batches on the GPU at once)")
    ap.add_argument("--serve-planners", type=int, default=2,
                    help="serving: planner threads (batches planned at once)")
    ap.add_argument("--tasks", choices=["both", "within", "across"], default="both")
    ap.add_argument("--plan-threads", type=int, default=1,
                    help="host threads planning the tasks of a step (1: in turn)")
    ap.add_argument("--streams", type=int, default=1,
                    help="CUDA streams that consecutive timed steps take in turn")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the BF16 / FP8, batched and serving parts of the default line")
    ap.add_argument("--ref-budget", type=float, default=5.0,
                    help="seconds of oracle CPU time per reference step / baseline sample")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload in ("batched", "serve"):  # one GPU each (replicas print nothing)
        line = (run_batched if args.workload == "batched" else run_serve)(args, rank, world)
        if rank == 0:
            print(json.dumps(line), flush=True)
    elif args.workload == "peaks":
        run_peaks(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
