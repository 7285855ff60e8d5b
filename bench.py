"""Benchmark of the B300 data-mapping-analysis hot path.

Default workload (one step): FP128 fingerprint of one 4 GiB buffer of random
bytes -- the largest size of the single-buffer bandwidth sweep -- through
odp_fingerprint, inputs resident in HBM (4 GiB > 126 MB L2, so no flush is
needed between steps).  The JSON line also carries the rest of the sweep,
the analysis throughput on the 50M-event iterative-solver trace, the batched
ragged form and the serving latencies when those parts are enabled.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the CPU oracle (the plain single-threaded
reference) on bounded samples of the same workload.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fingerprint GB/s vs HBM peak; M events/s analyzed; p99 event-to-finding latency"
BUF_BYTES = 4 << 30
SEED = 0x0DB2
# dram read+write bytes of one fp_tiles launch over 512 MiB from an ncu full
# capture of the default (8 warps, 2 bulk slots) kernel: 536.97 MB read +
# 4.02 MB written.
# Traffic grows with the bytes hashed: a launch over B bytes moves about
# B / 512 MiB times this.
FP_TILES_TRAFFIC_512MIB = 540.99e6
# DRAM read+write bytes of fp_tiles per algorithmic byte on a batch of 10^5
# ragged buffers (1.6 GiB, the batched workload's size distribution): 1,686.9 MB
# read + 4.4 MB written for 1,680.9 MB of buffers and per-buffer records.
# Traffic grows with the bytes hashed, so the 10^6-buffer call moves this
# ratio times its algorithmic bytes.
FP_BATCHED_TRAFFIC_RATIO = 1691.3e6 / 1680.9e6
# DRAM read+write bytes of one odp_analyze call on the 50,002,000-event
# iterative-solver trace, summed over its 124 launches (ncu, dram__bytes_read.sum
# + dram__bytes_write.sum, one pass per launch): 22.33 GB read + 11.03 GB written.
ANALYZE_TRAFFIC_PER_EVENT = 33.37e9 / 50_002_000


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class Clocks:
    """SM clock and clock-event-reason sampling (NVML, read-only) in a thread;
    summarised over the samples taken inside the timed window."""

    REASONS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20,
               "sw_power_cap": 0x4, "hw_power_brake_slowdown": 0x80}

    def __init__(self, device_index: int, period_s: float = 0.02):
        import threading

        self.dev = device_index
        self.period = period_s
        self.samples = []
        self.window = None
        self._stop = threading.Event()
        self._thread = threading.Thread(target=self._run, daemon=True)
        self.ok = False

    def _run(self):
        try:
            import pynvml

            pynvml.nvmlInit()
            h = pynvml.nvmlDeviceGetHandleByIndex(self.dev)
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(h, pynvml.NVML_CLOCK_SM)
            self.ok = True
            while not self._stop.is_set():
                t = time.perf_counter()
                sm = pynvml.nvmlDeviceGetClockInfo(h, pynvml.NVML_CLOCK_SM)
                try:
                    r = pynvml.nvmlDeviceGetCurrentClocksEventReasons(h)
                except Exception:
                    r = pynvml.nvmlDeviceGetCurrentClocksThrottleReasons(h)
                self.samples.append((t, sm, r))
                time.sleep(self.period)
        except Exception as e:  # NVML unusable: fall back to nvidia-smi
            self.err = repr(e)
            self._run_smi()

    def _run_smi(self):
        import subprocess

        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        bits = [0x8, 0x40, 0x20, 0x4]
        try:
            proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={q}",
                                     "--format=csv,noheader,nounits", "-lms", "50"],
                                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception as e:
            self.err += " / " + repr(e)
            return
        self.ok = True
        while not self._stop.is_set():
            line = proc.stdout.readline()
            if not line:
                break
            parts = [x.strip() for x in line.split(",")]
            try:
                sm, mx = float(parts[0]), float(parts[1])
            except (ValueError, IndexError):
                continue
            self.max_mhz = mx
            r = 0
            for b, v in zip(bits, parts[2:6]):
                if v.lower() == "active":
                    r |= b
            self.samples.append((time.perf_counter(), sm, r))
        proc.terminate()

    def __enter__(self):
        self._thread.start()
        time.sleep(0.1)
        return self

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __exit__(self, *a):
        self._stop.set()
        self._thread.join(timeout=5)

    def summary(self):
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                    "error": getattr(self, "err", "no samples")}
        inside = self.samples
        scope = "timed region"
        if self.window:
            w = [s for s in self.samples if self.window[0] <= s[0] <= self.window[1]]
            if len(w) >= 3:
                inside = w
            else:
                scope = "warm-up + timed region (timed region shorter than the sampling period)"
        reasons = set()
        for _, _, r in inside:
            for name, bit in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median([s[1] for s in inside]),
                "sm_max_mhz": self.max_mhz, "samples": len(inside), "scope": scope,
                "reasons": sorted(reasons)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = os.environ.get("ODP_BENCH_BACKEND",
                                 "nccl" if torch.cuda.is_available() else "gloo")
        dist.init_process_group(backend)
        return rank, world, local, dist
    return rank, world, local, None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def _reduce_device(dist):
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(dist, v):
    if dist is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, v):
    if dist is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------------- ours

def time_calls(fn, steps, warmup, stream):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    t0 = time.perf_counter()
    ev[0].record(stream)
    for i in range(steps):
        fn()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    time_calls.window = (t0, time.perf_counter())
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    total = ev[0].elapsed_time(ev[steps])
    return total, per


def run_ours(args):
    import torch

    rank, world, local, dist = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    import paper_2601_12713_b300 as odp
    from synth import gpu as sgpu, content

    stream = torch.cuda.current_stream()
    peak, peak_kind = peaks()
    parts = (set(args.only.split(",")) if args.only
             else {"fingerprint", "sweep", "plain_small", "batched", "analysis", "serving"})
    fp_bytes = args.fp_bytes
    result = {}
    if "fingerprint" in parts:
        buf = torch.empty(fp_bytes, dtype=torch.uint8, device="cuda")
        sgpu.fill(buf, content.RANDOM, SEED + rank)
        ptrs = torch.tensor([buf.data_ptr()], dtype=torch.int64, device="cuda")
        sizes = torch.tensor([fp_bytes], dtype=torch.int64, device="cuda")
        out = torch.empty((1, 2), dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()

        def step():
            odp.fingerprint(ptrs, sizes, out, stream)

        barrier(dist)
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            total_ms, per = time_calls(step, args.steps, args.warmup, stream)
            clk.mark(*time_calls.window)
        clocks = clk.summary()
        barrier(dist)
        t_max = max_over_ranks(dist, total_ms)
        bytes_all = sum_over_ranks(dist, float(fp_bytes) * args.steps)
        value = bytes_all / (t_max / 1e3) / 1e9
        per_launch_ms = statistics.mean(per)
        achieved = fp_bytes / (per_launch_ms / 1e3) / 1e9

        # end to end: pinned host bytes -> device -> fingerprint -> 16 B back
        e2e = None
        if not args.skip_e2e:
            host = torch.empty(fp_bytes, dtype=torch.uint8, pin_memory=True)
            host.copy_(buf)
            res_host = torch.empty((1, 2), dtype=torch.int64, pin_memory=True)

            def e2e_step():
                buf.copy_(host, non_blocking=True)
                odp.fingerprint(ptrs, sizes, out, stream)
                res_host.copy_(out, non_blocking=True)

            e_steps = max(3, min(args.steps, 10))
            e_total, _ = time_calls(e2e_step, e_steps, 2, stream)
            e_val = sum_over_ranks(dist, float(fp_bytes) * e_steps) / (
                max_over_ranks(dist, e_total) / 1e3) / 1e9
            e2e = {"value": round(e_val, 3), "unit": "GB/s", "h2d_bytes_per_step": fp_bytes,
                   "d2h_bytes_per_step": 16}
            del host
        result.update({
            "metric": METRIC,
            "value": round(value, 3),
            "unit": "GB/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(t_max / args.steps, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "u8",
            "data": "synthetic",
            "config": {
                "workload": "single-buffer fingerprint bandwidth sweep, largest size: one "
                            f"{fp_bytes >> 20} MiB buffer of seeded random bytes per step",
                "bytes_per_step_per_gpu": fp_bytes,
                "hash": "FP128 v1 (4 KiB chunks, left-balanced tree)",
                "l2": "inputs larger than the 126 MB L2: no flush between steps",
                "parallelism": f"replicas x{world}",
            },
            "clocks": clocks,
            "gpu_launches": args.steps,
            "roofline": {
                "bound": "hbm",
                "achieved": round(achieved, 2),
                "peak": peak,
                "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "peak_kind": f"{peak_kind} (copy read+write)",
                "traffic": args.traffic if args.traffic is not None else (
                    round(FP_TILES_TRAFFIC_512MIB * fp_bytes / (512 << 20))
                    if FP_TILES_TRAFFIC_512MIB else None),
                "traffic_source": "ncu capture of the 512 MiB case scaled by bytes",
                "kernel": "fp_tiles<8 warps, 2 bulk-copy slots> (CUDA events per "
                          "odp_fingerprint call; a one-buffer call is this single launch)",
                "algorithmic_bytes_per_launch": fp_bytes + 32,
            },
            "e2e": e2e,
        })
        if rank == 0:
            result["l2_resident"] = l2_resident(odp, buf, stream, peak, peak_kind)
        if rank == 0 and not args.skip_cpu:
            result["cpu_baseline"] = cpu_baseline_fp(buf)
        del buf
        torch.cuda.empty_cache()
    if rank == 0 and "sweep" in parts and not args.skip_sweep:
        result["sweep"] = sweep(odp, sgpu, content, stream)
    if "plain_small" in parts:
        result["plain_small"] = bench_plain_small(args, odp, dist, rank, stream, peak, peak_kind)
    if "batched" in parts:
        result["batched"] = bench_batched(args, odp, dist, rank, stream, peak, peak_kind)
    if "analysis" in parts:
        result["analysis"] = bench_analysis(args, odp, dist, rank, stream, peak, peak_kind)
    if "serving" in parts:
        result["serving"] = bench_serving(args, odp, dist, rank, stream)
        if args.serve_sweep:
            result["serving"]["rate_sweep"] = serving_rate_sweep(args, odp, rank)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def bench_batched(args, odp, dist, rank, stream, peak, peak_kind):
    """Ragged batch: 10^6 buffers, lognormal sizes (median 4 KiB), 16 GiB,
    40 % exact duplicates, one odp_fingerprint call (direct and replayed from
    a CUDA graph) against one launch per buffer on a sample."""
    import torch
    from synth import content, gpu as sgpu

    sizes, offs, seeds, dup_of = content.batched_ragged(seed=0x0DB3 + rank, n=args.batched_n,
                                                        total=args.batched_bytes)
    n = sizes.size
    total = int(sizes.sum())
    arena = torch.empty(int(offs[-1] + sizes[-1]) + 64, dtype=torch.uint8, device="cuda")
    sgpu.fill_many(arena, offs, sizes, seeds)
    ptrs = torch.from_numpy(arena.data_ptr() + offs).cuda()
    sz = torch.from_numpy(sizes).cuda()
    out = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    if args.no_autotune:
        # the schedule cached by an earlier tuning run (ODP_AUTOTUNE_CACHE), or
        # the defaults: lets a profiler see the kernel the timed calls use
        sched, tuned_ms = ("cached",), 0.0
    else:
        sched, tuned_ms = odp.autotune_fingerprint(ptrs, sz, out, reps=2, stream=stream)
    steps = max(3, min(args.steps, 10))
    d_total, d_per = time_calls(lambda: odp.fingerprint(ptrs, sz, out, stream), steps,
                                args.warmup, stream)

    # the same call replayed from a CUDA graph (scratch warmed on the capture stream)
    cap = torch.cuda.Stream()
    cap.wait_stream(stream)
    with torch.cuda.stream(cap):
        odp.fingerprint(ptrs, sz, out, cap)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        odp.fingerprint(ptrs, sz, out, cap)
    g_total, g_per = time_calls(graph.replay, steps, 2, stream)
    g_max = max_over_ranks(dist, g_total)
    value = sum_over_ranks(dist, float(total) * steps) / (g_max / 1e3) / 1e9
    direct = sum_over_ranks(dist, float(total) * steps) / (
        max_over_ranks(dist, d_total) / 1e3) / 1e9
    fps = out.cpu().numpy().view(np.uint64).copy()

    # one launch per buffer on a sample, captured in a graph (no host gaps)
    S = min(n, args.per_buffer_sample)
    s_bytes = int(sizes[:S].sum())
    out_s = torch.empty((S, 2), dtype=torch.int64, device="cuda")
    with torch.cuda.stream(cap):
        odp.fingerprint(ptrs[:1], sz[:1], out_s[:1], cap)
    torch.cuda.synchronize()
    g1 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g1, stream=cap):
        for i in range(S):
            odp.fingerprint(ptrs[i:i + 1], sz[i:i + 1], out_s[i:i + 1], cap)
    p_total, _ = time_calls(g1.replay, 3, 1, stream)
    per_buffer = s_bytes * 3 / (p_total / 1e3) / 1e9
    same_ok = bool(np.array_equal(out_s.cpu().numpy().view(np.uint64), fps[:S]))
    b_total, _ = time_calls(lambda: odp.fingerprint(ptrs[:S], sz[:S], out_s, stream), 3, 2,
                            stream)
    batched_sample = s_bytes * 3 / (b_total / 1e3) / 1e9
    del g1

    # sampled parity against the oracle, and duplicate consistency
    parity = None
    if rank == 0:
        import oracle

        rng = np.random.default_rng(12)
        idx = rng.choice(n, 200, replace=False)
        idx = np.concatenate([idx, np.argsort(sizes)[-3:]])
        ok = True
        for i in idx:
            data = content.bytes_of(content.RANDOM, int(seeds[i]), int(sizes[i]))
            ok &= oracle.fp128(data) == (int(fps[i, 0]), int(fps[i, 1]))
        d = np.flatnonzero(dup_of >= 0)
        dup_ok = bool(np.array_equal(fps[d], fps[dup_of[d]]))
        parity = {"sampled_buffers": int(idx.size), "oracle_equal": bool(ok),
                  "duplicates_equal": dup_ok, "distinct_fps": int(np.unique(
                      fps[dup_of < 0], axis=0).shape[0]), "originals": int((dup_of < 0).sum())}
    per_ms = statistics.mean(g_per)
    achieved = total / (per_ms / 1e3) / 1e9
    res = {
        "metric": "fingerprint GB/s (batched ragged, one call)",
        "value": round(value, 2),
        "unit": "GB/s",
        "ms_per_step": round(g_max / steps, 4),
        "direct_call_gbs": round(direct, 2),
        "config": {"workload": f"{n} buffers, lognormal sizes (median 4 KiB, sigma sqrt(2 ln 4)) "
                               f"clipped to [1 B, 256 MiB], {total} bytes, 40 % duplicates, "
                               "16-byte-aligned arena", "buffers": n, "bytes": total,
                   "autotuned_schedule": list(sched), "autotune_ms": round(tuned_ms, 4)},
        "per_buffer_launches": {"buffers": S, "bytes": s_bytes, "gbs": round(per_buffer, 2),
                                "batched_same_buffers_gbs": round(batched_sample, 2),
                                "speedup": round(batched_sample / per_buffer, 2),
                                "identical_results": same_ok,
                                "note": "one odp_fingerprint launch per buffer, all captured in "
                                        "one CUDA graph (no host launch gaps)"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "peak_kind": f"{peak_kind} (copy read+write)",
                     "algorithmic_bytes_per_launch": total + 32 * n,
                     "traffic": round(FP_BATCHED_TRAFFIC_RATIO * (total + 32 * n)),
                     "traffic_source": "ncu capture of fp_tiles on a 10^5-buffer, 1.6 GiB batch "
                                       "of the same size distribution, scaled by the "
                                       "algorithmic bytes"},
        "parity": parity,
    }
    if rank == 0 and not args.skip_cpu:
        import oracle

        host = arena[: int(offs[min(n - 1, 40000)])].cpu().numpy()
        k = int(np.searchsorted(offs, host.size)) - 1
        t0 = time.perf_counter()
        oracle.fp128_many(host, offs[:k], sizes[:k])
        dt = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": round(int(sizes[:k].sum()) / dt / 1e9, 4), "unit": "GB/s",
                               "cores": 1, "kind": "oracle",
                               "sample": f"first {k} buffers of the batch "
                                         f"({int(sizes[:k].sum())} bytes)"}
    del arena, out, out_s, graph
    torch.cuda.empty_cache()
    return res


def bench_plain_small(args, odp, dist, rank, stream, peak, peak_kind):
    """Plain small workload: the 4,000-data-op trace over 128 host buffers
    (plus its kernel events), every transfer's payload resident in HBM.  A
    step fingerprints every transfer and runs Algorithms 1-5 over the log:

      plain      one odp_fingerprint launch per transfer, its output written
                 straight into the transfer's record, then odp_analyze;
      plain_one  the same through odp_fingerprint_one;
      batched    odp_fingerprint_log (every transfer in one call) and
                 odp_analyze;
      serving    the trace submitted to an odp_server that fingerprints the
                 payloads and streams the findings, flushed and polled.

    All forms must give the oracle's findings.  The one-launch-per-transfer
    forms are timed as the host issues them and replayed from a CUDA graph
    (device time only)."""
    import torch
    from synth import content, gpu as sgpu, traces

    b = traces.plain_small(seed=0x0DB1 + rank)
    ev = b.events.copy()
    ev["fp_lo"] = 0
    ev["fp_hi"] = 0
    n = ev.size
    xfer = np.flatnonzero(np.isin(ev["kind"], [2, 3, 4]))
    sizes = ev["bytes"][xfer].astype(np.int64)
    offs = np.concatenate([[0], np.cumsum((sizes + 255) // 256 * 256)[:-1]]).astype(np.int64)
    payload_bytes = int(sizes.sum())
    arena = torch.empty(int(offs[-1] + sizes[-1]) + 256, dtype=torch.uint8, device="cuda")
    sgpu.fill_many(arena, offs, sizes, b.payload_seed[xfer].astype(np.uint64))
    ptr_all = np.zeros(n, dtype=np.int64)
    ptr_all[xfer] = arena.data_ptr() + offs
    d_ptrs = torch.from_numpy(ptr_all).cuda()
    x_ptrs = torch.from_numpy(arena.data_ptr() + offs).cuda()
    x_sizes = torch.from_numpy(sizes).cuda()
    ev_host = torch.from_numpy(ev.view(np.uint8).reshape(-1).copy()).pin_memory()
    d_ev = ev_host.cuda()
    out = odp.Findings(6 * n)
    fp_views = [d_ev[64 * int(i) + 40:64 * int(i) + 56].view(torch.int64) for i in xfer]
    p_views = [x_ptrs[k:k + 1] for k in range(xfer.size)]
    s_views = [x_sizes[k:k + 1] for k in range(xfer.size)]
    h_ptrs = [int(arena.data_ptr() + o) for o in offs]
    h_sizes = [int(v) for v in sizes]

    def plain(s_):
        for k in range(xfer.size):
            odp.fingerprint(p_views[k], s_views[k], fp_views[k], s_)
        odp.analyze(d_ev, n, out, s_)

    def plain_one(s_):
        for k in range(xfer.size):
            odp.fingerprint_one(h_ptrs[k], h_sizes[k], fp_views[k], s_)
        odp.analyze(d_ev, n, out, s_)

    def batched(s_):
        odp.fingerprint_log(d_ev, n, d_ptrs, s_)
        odp.analyze(d_ev, n, out, s_)

    # the oracle's findings for this trace, from the oracle's own fingerprints
    import oracle

    host_payloads = arena.cpu().numpy()
    t0 = time.perf_counter()
    fps_o = oracle.fp128_many(host_payloads, offs, sizes)
    ev_o = ev.copy()
    ev_o["fp_lo"][xfer], ev_o["fp_hi"][xfer] = fps_o[:, 0], fps_o[:, 1]
    o = oracle.analyze(ev_o)
    cpu_s = time.perf_counter() - t0

    def same_as_oracle():
        r = out.to_host()
        ok = (r["status"] == o.status and r["count"] == o.count and r["summary"] == o.summary
              and np.array_equal(r["findings"].view(np.uint8), o.findings.view(np.uint8))
              and np.array_equal(r["sites"].view(np.uint8), o.sites.view(np.uint8)))
        return bool(ok and np.array_equal(d_ev.cpu().numpy(), ev_o.view(np.uint8).reshape(-1)))

    steps = max(3, min(args.steps, 10))
    forms = {}
    for name, fn in (("plain", plain), ("plain_one", plain_one), ("batched", batched)):
        d_ev.copy_(ev_host)
        total, _ = time_calls(lambda: fn(stream), steps, args.warmup, stream)
        t_max = max_over_ranks(dist, total)
        row = {"ms_per_step": round(t_max / steps, 4),
               "events_per_s": round(sum_over_ranks(dist, float(n) * steps) / (t_max / 1e3), 1),
               "identical_to_oracle": same_as_oracle()}
        # device time without the host's launch gaps: the whole step in a graph
        cap = torch.cuda.Stream()
        cap.wait_stream(stream)
        with torch.cuda.stream(cap):
            fn(cap)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            fn(cap)
        d_ev.copy_(ev_host)
        g_total, _ = time_calls(g.replay, steps, 2, stream)
        g_max = max_over_ranks(dist, g_total)
        row["graph_ms_per_step"] = round(g_max / steps, 4)
        row["graph_events_per_s"] = round(
            sum_over_ranks(dist, float(n) * steps) / (g_max / 1e3), 1)
        row["graph_identical_to_oracle"] = same_as_oracle()
        if name != "batched":
            row["launches_per_step"] = int(xfer.size) + 1
        del g
        forms[name] = row

    # serving: one producer submits the whole trace; the server fingerprints
    # every payload and streams the findings
    srv_rows = []
    want = o.findings[np.lexsort((o.findings["partner"], o.findings["event"],
                                  o.findings["kind"]))]
    payload_arg = ptr_all.astype(np.uint64)
    for _ in range(3):
        srv = odp.Server(n_slots=4, device_budget_bytes=4 << 30, max_events=1 << 16,
                         max_batch_events=4096, max_producers=4, watermark_timeout_us=50_000)
        srv.attach(0)
        t0 = time.perf_counter()
        srv.submit(ev, payload_arg)
        srv.flush()
        got = srv.poll(1 << 20)
        dt = time.perf_counter() - t0
        got = got[np.lexsort((got["partner"], got["event"], got["kind"]))]
        srv_rows.append((dt, bool(got.size == want.size and np.array_equal(
            got.view(np.uint8), want.view(np.uint8)))))
        srv.close()
    srv_s = statistics.median([r[0] for r in srv_rows])
    forms["serving"] = {"ms_per_step": round(srv_s * 1e3, 4),
                        "events_per_s": round(n / srv_s, 1),
                        "identical_to_oracle": all(r[1] for r in srv_rows),
                        "note": "wall time from submit to the last finding polled (host "
                                "clock), median of 3 fresh servers"}

    # end to end through the public API: events and payloads from pinned host
    # memory, one batched step, the summary words back
    host_arena = torch.empty(arena.numel(), dtype=torch.uint8, pin_memory=True)
    host_arena.copy_(arena)
    small_host = torch.empty(out.small.numel(), dtype=torch.int64, pin_memory=True)

    def e2e_step():
        arena.copy_(host_arena, non_blocking=True)
        d_ev.copy_(ev_host, non_blocking=True)
        batched(stream)
        small_host.copy_(out.small, non_blocking=True)

    e_total, _ = time_calls(e2e_step, steps, 2, stream)
    e_val = sum_over_ranks(dist, float(n) * steps) / (max_over_ranks(dist, e_total) / 1e3) / 1e6

    r = out.to_host()
    alg_bytes = payload_bytes + 64 * n + 48 * r["count"] + 32 * r["n_sites"]
    best = forms["batched"]["ms_per_step"]
    plain_dev = forms["plain"]["graph_ms_per_step"]
    res = {
        "metric": "M events/s analyzed (every transfer fingerprinted, then Alg. 1-5)",
        "value": round(forms["batched"]["events_per_s"] / 1e6, 4),
        "unit": "M events/s",
        "ms_per_step": best,
        "config": {"workload": "plain small: 128 host buffers (log-uniform 4 KiB..1 MiB), 1,000 "
                               "map cycles, 4,000 data ops + kernels, 30 % resent contents, "
                               "10 % round trips, 5 % re-allocations, payloads resident in HBM",
                   "events": n, "transfers": int(xfer.size), "payload_bytes": payload_bytes,
                   "findings": r["count"],
                   "counts": [r["summary"][f"count{k}"] for k in range(1, 6)]},
        "forms": forms,
        "speedup_vs_plain": {
            "batched_vs_plain_host_issued": round(forms["plain"]["ms_per_step"] / best, 2),
            "batched_vs_plain_graph": round(plain_dev / best, 2),
            "batched_vs_plain_one_graph": round(forms["plain_one"]["graph_ms_per_step"] / best, 2),
            "batched_graph_vs_plain_graph": round(
                plain_dev / forms["batched"]["graph_ms_per_step"], 2),
            "serving_vs_plain_host_issued": round(
                forms["plain"]["ms_per_step"] / forms["serving"]["ms_per_step"], 2)},
        "roofline": {"bound": "hbm", "achieved": round(alg_bytes / (best / 1e3) / 1e9, 2),
                     "peak": peak, "unit": "GB/s",
                     "frac": round(alg_bytes / (best / 1e3) / 1e9 / peak, 4),
                     "peak_kind": f"{peak_kind} (copy read+write)",
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "note": "one batched step (odp_fingerprint_log + odp_analyze): payload "
                             "bytes read once, 64 B per event, 48 B per finding, 32 B per "
                             "site row, over the step's CUDA-event time"},
        "e2e": {"value": round(e_val, 4), "unit": "M events/s",
                "h2d_bytes_per_step": int(arena.numel()) + 64 * n,
                "d2h_bytes_per_step": 8 * out.small.numel()},
        "cpu_baseline": {"value": round(n / cpu_s / 1e6, 6), "unit": "M events/s", "cores": 1,
                         "host_cores": os.cpu_count(), "kind": "oracle",
                         "sample": "the whole trace: FP128 of every transfer's payload, then "
                                   "Alg. 1-5, single-threaded oracle"},
    }
    del arena, d_ev, out, host_arena
    torch.cuda.empty_cache()
    return res


def serving_rate_sweep(args, odp, rank):
    """Latency and sustained rate of the serving loop at higher offered
    rates (same producers and payloads, shorter runs so the log fits)."""
    import torch
    from synth import content, gpu as sgpu, load

    pool_bytes = 1 << 30
    pool = torch.empty(pool_bytes, dtype=torch.uint8, device="cuda")
    sgpu.fill(pool, content.RANDOM, 0x0DB6 + rank)
    torch.cuda.synchronize()
    rows = []
    for rate in [float(x) for x in args.serve_sweep.split(",")]:
        cap = 1 << 23
        secs = min(args.serve_sweep_seconds, 0.9 * cap / rate)  # the log holds the run
        srv = odp.Server(n_slots=4, device_budget_bytes=8 << 30, max_events=cap,
                         max_batch_events=8192, max_producers=128, watermark_timeout_us=50_000)
        lg = load.Load(64, rate, secs, 0x0DB6 + rank, pool.data_ptr(), pool_bytes, 256, 64 << 20)
        n = lg.run(srv, announce=args.serve_stamp == "begin")
        srv.flush()
        st = srv.stats()
        span_s = (st["last_done_ns"] - st["first_submit_ns"]) / 1e9
        rows.append({"offered_events_per_s": rate, "seconds": round(secs, 2), "events": n,
                     "sustained_events_per_s": round(st["events_processed"] / span_s, 1),
                     "p50_ms": round(st["latency_p50_ns"] / 1e6, 3),
                     "p99_ms": round(st["latency_p99_ns"] / 1e6, 3),
                     "before_launch_p99_ms": round(st["queue_p99_ns"] / 1e6, 3),
                     "batches": st["batches"], "late_events": st["late_events"],
                     "stream_overflow": st["stream_overflow"]})
        srv.close()
        lg.close()
    del pool
    torch.cuda.empty_cache()
    return rows


def bench_serving(args, odp, dist, rank, stream):
    """Serving loop: 64 producer threads, Poisson arrivals at an aggregate
    2e5 events/s, payloads log-uniform 256 B .. 64 MiB viewed in a 1 GiB
    device content pool, device state budget 8 GiB."""
    import torch
    from synth import content, gpu as sgpu, load

    pool_bytes = 1 << 30
    pool = torch.empty(pool_bytes, dtype=torch.uint8, device="cuda")
    sgpu.fill(pool, content.RANDOM, 0x0DB5 + rank)
    torch.cuda.synchronize()
    rate = args.serve_rate
    secs = args.serve_seconds
    max_events = 1 << 23
    srv = odp.Server(n_slots=args.serve_slots, device_budget_bytes=8 << 30, max_events=max_events,
                     max_batch_events=8192, max_producers=128, watermark_timeout_us=50_000,
                     batch_interval_us=args.serve_interval_us)
    lg = load.Load(64, rate, secs, 0x0DB5 + rank, pool.data_ptr(), pool_bytes, 256, 64 << 20)
    n = lg.run(srv, announce=args.serve_stamp == "begin")
    srv.flush()
    st = srv.stats()
    streamed = srv.poll(1 << 24)
    span_s = (st["last_done_ns"] - st["first_submit_ns"]) / 1e9
    sustained = st["events_processed"] / span_s
    # offline batched form over the same merged log: fingerprint every
    # transfer in one call, then odp_analyze
    log = odp.log_tensor(srv, n)
    ev = log.cpu().numpy().view(odp.EVENT_DTYPE).copy()
    prod, seq = srv.origin(n)
    is_x = np.isin(ev["kind"], [2, 3, 4])
    idx = np.flatnonzero(is_x)
    views = np.array([lg.payload(lg.thread_of(ev["host_addr"][i]), int(seq[i])) for i in idx],
                     dtype=np.int64).reshape(-1, 2)
    ptrs = torch.tensor(pool.data_ptr() + views[:, 0], dtype=torch.int64, device="cuda")
    sizes = torch.tensor(views[:, 1], dtype=torch.int64, device="cuda")
    fps = torch.empty((idx.size, 2), dtype=torch.int64, device="cuda")
    out = odp.Findings(6 * n)

    def offline():
        odp.fingerprint(ptrs, sizes, fps, stream)
        odp.analyze(log, n, out, stream)

    o_total, _ = time_calls(offline, 3, 1, stream)
    offline_rate = n / (o_total / 3 / 1e3)
    g = out.to_host()
    same_fp = bool(np.array_equal(fps.cpu().numpy().view(np.uint64),
                                  np.stack([ev["fp_lo"][idx], ev["fp_hi"][idx]], axis=1)))
    off = g["findings"]
    st_sorted = streamed[np.lexsort((streamed["partner"], streamed["event"], streamed["kind"]))]
    same_findings = bool(st_sorted.size == off.size and
                         np.array_equal(st_sorted.view(np.uint8), off.view(np.uint8)))
    res = {
        "metric": "p99 event-to-finding latency",
        "value": round(st["latency_p99_ns"] / 1e6, 3),
        "unit": "ms",
        "higher_is_better": False,
        "p50_ms": round(st["latency_p50_ns"] / 1e6, 3),
        "max_ms": round(st["latency_max_ns"] / 1e6, 3),
        "before_launch_p50_ms": round(st["queue_p50_ns"] / 1e6, 3),
        "before_launch_p99_ms": round(st["queue_p99_ns"] / 1e6, 3),
        "sustained_events_per_s": round(sustained, 1),
        "offline_batched_events_per_s": round(offline_rate, 1),
        "config": {"workload": f"64 producer threads, Poisson arrivals, {rate:.0f} events/s "
                               f"aggregate for {secs} s, payloads log-uniform 256 B..64 MiB "
                               f"(views of a 1 GiB device pool), {args.serve_slots} slots, 8192-event batches, "
                               "8 GiB device budget", "events": n, "batches": st["batches"],
                   "start_stamps": ("odp_server_begin (the merge waits only for open events)"
                                    if args.serve_stamp == "begin" else
                                    "by each producer (the merge waits for each one's next event)"),
                   "transfers": int(idx.size), "payload_bytes": int(views[:, 1].sum())},
        "findings_streamed": int(streamed.size),
        "streamed_equal_offline": same_findings,
        "fingerprints_alone_equal_mix": same_fp,
        "offline_counts": [g["summary"][f"count{k}"] for k in range(1, 6)],
        "late_events": st["late_events"],
        "latency_definition": "submit call of the completing event -> finding in the poll queue",
    }
    srv.close()
    lg.close()
    del pool, log, out, fps
    torch.cuda.empty_cache()
    return res


def bench_analysis(args, odp, dist, rank, stream, peak, peak_kind):
    """odp_analyze on the iterative-solver trace (2,000 iterations x 25,000
    arrays, 6,250 mapped per iteration: 5e7 data-op events + 2,000 kernels)."""
    import torch
    from synth import traces

    n_iter = args.analysis_iters
    b = traces.iterative_solver(seed=0x0DB4 + rank, n_iter=n_iter)
    traces.fill_fp_from_content(b)
    n = b.events.size
    host = torch.from_numpy(b.events.view(np.uint8).reshape(-1)).pin_memory()
    ev = host.to("cuda")
    out = odp.Findings(n)
    steps = max(3, min(args.steps, 10))

    def step():
        odp.analyze(ev, n, out, stream)

    total_ms, per = time_calls(step, steps, args.warmup, stream)
    t_max = max_over_ranks(dist, total_ms)
    ev_all = sum_over_ranks(dist, float(n) * steps)
    value = ev_all / (t_max / 1e3) / 1e6
    r = out.to_host()
    findings = r["count"]
    alg_bytes = 64 * n + 48 * findings + 32 * r["n_sites"]
    per_ms = statistics.mean(per)
    achieved = alg_bytes / (per_ms / 1e3) / 1e9

    small_host = torch.empty(out.small.numel(), dtype=torch.int64, pin_memory=True)

    def e2e_step():
        ev.copy_(host, non_blocking=True)
        odp.analyze(ev, n, out, stream)
        small_host.copy_(out.small, non_blocking=True)

    e_steps = 3
    e_total, _ = time_calls(e2e_step, e_steps, 1, stream)
    e_val = sum_over_ranks(dist, float(n) * e_steps) / (max_over_ranks(dist, e_total) / 1e3) / 1e6
    res = {
        "metric": "M events/s analyzed",
        "value": round(value, 2),
        "unit": "M events/s",
        "ms_per_step": round(t_max / steps, 3),
        "steps": steps,
        "config": {"workload": f"iterative offload solver trace: {n_iter} iterations x 25,000 "
                               "float64 arrays, 6,250 mapped per iteration, p(change)=0.2, "
                               "500 sites", "events": n, "findings": findings,
                   "counts": [r["summary"][f"count{k}"] for k in range(1, 6)],
                   "status": r["status"]},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_kind": f"{peak_kind} (copy read+write)",
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "traffic": round(ANALYZE_TRAFFIC_PER_EVENT * n),
                     "traffic_source": "ncu capture of one call on this 50,002,000-event trace "
                                       "(all 124 launches), per event times the events",
                     "note": "whole odp_analyze call against the bytes the method must read "
                             "and write: 64 B per event, 48 B per finding, 32 B per site row"},
        "e2e": {"value": round(e_val, 2), "unit": "M events/s", "h2d_bytes_per_step": 64 * n,
                "d2h_bytes_per_step": 8 * out.small.numel()},
    }
    # the same trace with 3 % of the iterations' kernels moved to another
    # device: Alg. 4 and 5 then emit (unused allocations and transfers)
    traces.skip_kernels(b.events, 0.03, 0x0DB4 + rank)
    host.copy_(torch.from_numpy(b.events.view(np.uint8).reshape(-1)))
    ev.copy_(host)
    u_total, u_per = time_calls(step, steps, args.warmup, stream)
    u_max = max_over_ranks(dist, u_total)
    ru = out.to_host()
    u_bytes = 64 * n + 48 * ru["count"] + 32 * ru["n_sites"]
    u_achieved = u_bytes / (statistics.mean(u_per) / 1e3) / 1e9
    res["with_unused"] = {
        "value": round(sum_over_ranks(dist, float(n) * steps) / (u_max / 1e3) / 1e6, 2),
        "unit": "M events/s", "ms_per_step": round(u_max / steps, 3),
        "config": {"workload": "the same trace with 3 % of the iterations' kernels on another "
                               "device (their allocations unused, their to-device transfers "
                               "overwritten unused in the next iteration)",
                   "kernels_moved": int((b.events["dst_dev"][b.events["kind"] == 6] == 1).sum()),
                   "findings": ru["count"],
                   "counts": [ru["summary"][f"count{k}"] for k in range(1, 6)],
                   "status": ru["status"]},
        "roofline": {"bound": "hbm", "achieved": round(u_achieved, 2), "peak": peak,
                     "unit": "GB/s", "frac": round(u_achieved / peak, 4),
                     "algorithmic_bytes_per_launch": u_bytes},
    }
    if rank == 0 and not args.skip_cpu:
        import oracle

        sb = traces.iterative_solver(seed=0x0DB4, n_iter=20)
        traces.fill_fp_from_content(sb)
        t0 = time.perf_counter()
        o = oracle.analyze(sb.events)
        dt = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": round(sb.events.size / dt / 1e6, 4), "unit": "M events/s",
                               "cores": 1, "kind": "oracle",
                               "sample": f"first 20 iterations of the same trace shape "
                                         f"({sb.events.size} events), status {o.status}"}
    del ev, out, host
    torch.cuda.empty_cache()
    return res


def sweep(odp, sgpu, content, stream):
    import torch

    rows = []
    for variant_name in ("random", "zero", "page"):
        v = content.VARIANTS[variant_name]
        for k in range(9):
            size = (64 << 10) * (4 ** k)
            buf = torch.empty(size, dtype=torch.uint8, device="cuda")
            sgpu.fill(buf, v, SEED + k)
            ptrs = torch.tensor([buf.data_ptr()], dtype=torch.int64, device="cuda")
            sizes = torch.tensor([size], dtype=torch.int64, device="cuda")
            out = torch.empty((1, 2), dtype=torch.int64, device="cuda")
            reps = 20 if size <= (64 << 20) else 5
            _, per = time_calls(lambda: odp.fingerprint(ptrs, sizes, out, stream), reps, 3, stream)
            med = statistics.median(per)
            # the same buffer through odp_fingerprint_one (host-side pointer and
            # size, launch sized to the buffer)
            _, per1 = time_calls(lambda: odp.fingerprint_one(buf.data_ptr(), size, out, stream),
                                 reps, 3, stream)
            med1 = statistics.median(per1)
            row = {"variant": variant_name, "bytes": size,
                   "gbs": round(size / (med / 1e3) / 1e9, 2), "ms": round(med, 4),
                   "one_gbs": round(size / (med1 / 1e3) / 1e9, 2), "one_ms": round(med1, 4)}
            if size <= (16 << 20):
                # small calls are bound by the host's launch rate: also the
                # device time per call, 20 calls replayed from a CUDA graph
                for key, fn in (("graph_ms", lambda s_: odp.fingerprint(ptrs, sizes, out, s_)),
                                ("one_graph_ms",
                                 lambda s_: odp.fingerprint_one(buf.data_ptr(), size, out, s_))):
                    cap = torch.cuda.Stream()
                    cap.wait_stream(stream)
                    with torch.cuda.stream(cap):
                        fn(cap)
                    torch.cuda.synchronize()
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g, stream=cap):
                        for _ in range(20):
                            fn(cap)
                    tot, _ = time_calls(g.replay, 5, 2, stream)
                    row[key] = round(tot / 5 / 20, 5)
            rows.append(row)
            del buf
    return rows


def l2_resident(odp, buf, stream, peak, peak_kind):
    """The hash kernel's ceiling away from HBM: one call over 128 aliases of
    one 32 MiB slice (4 GiB hashed, the slice stays in the 126 MB L2).  A rate
    well above the HBM peak shows that the ALU does not bind the HBM-sized
    case."""
    import torch

    sl, k = 32 << 20, 128
    ptrs = torch.full((k,), buf.data_ptr(), dtype=torch.int64, device="cuda")
    sizes = torch.full((k,), sl, dtype=torch.int64, device="cuda")
    out = torch.empty((k, 2), dtype=torch.int64, device="cuda")
    total, _ = time_calls(lambda: odp.fingerprint(ptrs, sizes, out, stream), 10, 3, stream)
    gbs = sl * k * 10 / (total / 1e3) / 1e9
    o = out.cpu().numpy()
    return {"gbs": round(gbs, 1), "vs_hbm_peak": round(gbs / peak, 3),
            "peak_kind": f"{peak_kind} (copy read+write)",
            "input": "128 aliases of one 32 MiB slice of the benchmark buffer in one call",
            "identical_fingerprints": bool((o == o[0]).all())}


def cpu_baseline_fp(buf):
    import concurrent.futures

    import oracle

    sample = 1 << 30
    host = buf[:sample].cpu().numpy()
    oracle.build()
    t0 = time.perf_counter()
    oracle.fp128(host)
    dt = time.perf_counter() - t0
    # the same oracle function on every host core (one slice per thread; the
    # oracle call releases the interpreter lock)
    threads = os.cpu_count() or 1
    step = sample // threads
    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        t1 = time.perf_counter()
        list(ex.map(lambda i: oracle.fp128(host[i * step:(i + 1) * step]), range(threads)))
        dt_all = time.perf_counter() - t1
    return {"value": round(sample / dt / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "first 1 GiB of the 4 GiB random buffer, FP128 by the single-threaded oracle",
            "all_cores": {"value": round(step * threads / dt_all / 1e9, 4), "unit": "GB/s",
                          "threads": threads,
                          "sample": "the same 1 GiB in one slice per host thread"}}


# ---------------------------------------------------------------- reference

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from synth import content

    oracle.build()
    sample = 256 << 20
    data = content.bytes_of(content.RANDOM, SEED, sample)
    for _ in range(args.warmup):
        oracle.fp128(data[: 1 << 20])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fp128(data)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sample * args.steps / total / 1e9
    result = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 4),
        "unit": "GB/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(total / args.steps * 1e3, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {
            "workload": "single-buffer fingerprint bandwidth sweep, largest size: one 4 GiB "
                        "buffer of seeded random bytes per step",
            "parallelism": "cpu oracle, 1 thread",
        },
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "256 MiB of the workload's random bytes per step"},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(result), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-sweep", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--only", default="", help="comma list of parts: fingerprint,sweep,plain_small,batched,analysis,"
                    "serving")
    ap.add_argument("--fp-bytes", type=int, default=BUF_BYTES)
    ap.add_argument("--analysis-iters", type=int, default=2000)
    ap.add_argument("--batched-n", type=int, default=1_000_000)
    ap.add_argument("--batched-bytes", type=int, default=16 << 30)
    ap.add_argument("--per-buffer-sample", type=int, default=20_000)
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--serve-rate", type=float, default=200_000.0)
    ap.add_argument("--serve-slots", type=int, default=4, help="batches in flight at most")
    ap.add_argument("--serve-interval-us", type=int, default=50,
                    help="batcher polling period of the serving loop")
    ap.add_argument("--serve-sweep", default="",
                    help="comma list of offered rates (events/s) for an extra latency sweep")
    ap.add_argument("--serve-sweep-seconds", type=float, default=5.0)
    ap.add_argument("--serve-stamp", default="begin", choices=["begin", "self"],
                    help="producers open each event with odp_server_begin (the merge waits only "
                         "for open events) or stamp it themselves (the merge waits for every "
                         "producer's next event)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched part: no tuning; use the schedule cached in ODP_AUTOTUNE_CACHE")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the dominant kernel, if captured")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
