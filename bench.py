"""Benchmark of the batched DP alignment path on GB300.

Workload (one step = one anyseq_align_batch call over the whole batch):
262,144 short-read pairs, query 100-250 bp, target = query with 4 %
substitutions, 1 % indels and 20-bp flanks; semi-global alignment with affine
gaps (+1 / -4 / open -6 / extend -1), int16x2 lanes, score and optimum cell.
The barrier and the max over ranks are timing only.

Under torchrun the ranks split one global batch of N x 262,144 pairs by the
library's length-balanced round-robin partition (anyseq_shard_plan), so the
work per GPU stays fixed (weak scaling); after the timed region rank 0
gathers every pair's record in the caller's order (the path's one exchange).

Prints one JSON line. ``value`` is cell updates per second (GCUPS) with inputs
resident in device memory; ``e2e`` is the same metric through the C ABI with
pinned host buffers, host-device copies inside the timed region; ``roofline``
is the DP kernel's cell rate against the integer-issue bound
SMs x clock x I_SM / I_alg. I_alg = 3.5 algorithmic ops per cell for int16x2
affine (7 for int32), fixed before measuring. I_SM is the per-SM issue rate of
the fused cell's instruction mix on the SM's pipes: per lane-word the cell
issues 4 half-rate ops (byte permute, two DPX add-max, one three-input max:
64 lanes per clock per SM, measured) and 2 full-rate 32-bit adds (128 lanes
per clock), under the SM's issue limit of 128 lane-instructions per clock, so
I_SM = 6 / max(4/64, 2/128, 6/128) = 96 lane-ops per clock;
``cpu_baseline`` is the CPU oracle on the host cores on a bounded sample.
``--impl reference`` times the CPU oracle itself on the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "GCUPS & % of int-issue roofline; pairs/s learned-band vs full DP, scores exact"
WORKLOAD = "short_reads_262144_semiglobal_affine"
SCORING = (1, -4, -6, -1)
MODE = 2  # semi-global
I_ALG = 3.5  # algorithmic integer ops per cell, int16x2 affine (fixed before measuring)
I_ALG32 = 7.0  # the same for 32-bit lanes
# Issue rates per SM in lanes per clock, measured on GB300 (sm_103) with
# dependent-chain throughput probes: DPX add-max, three-input max and byte
# permute run at half rate; 32-bit IADD at full rate; the SM issues at most
# 4 sub-partitions x 32 lanes per clock.
HALF_RATE, FULL_RATE, ISSUE_RATE = 64, 128, 128
# instruction mix of the fused cell per lane-word: byte permute (sigma'),
# add-max (F), three-input max (H), add-max (E) at half rate; the diagonal
# add and H + open + extend at full rate
CELL_MIX = {"half": 4, "full": 2}
NOMINAL_LANE_OPS = 128  # 4 SM sub-partitions x 32 lanes


def lane_ops_per_clk(mix=CELL_MIX) -> float:
    """I_SM: ops of the mix / the clocks its busiest pipe (or the issue port) needs."""
    ops = mix["half"] + mix["full"]
    clocks = max(mix["half"] / HALF_RATE, mix["full"] / FULL_RATE, ops / ISSUE_RATE)
    return ops / clocks


LANE_OPS_PER_CLK = lane_ops_per_clk()  # 96
L2_BYTES = 129 * 2**20


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


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x: float, device) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(ws, x: float, device) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms. start() returns
    once the sampler has printed its first line; begin() marks the start of the
    timed region; stop() keeps the samples taken after the mark (all of them if
    the region was too short for one)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.mark = 0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t0 = time.perf_counter()
        while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 3.0:
            time.sleep(0.005)

    def begin(self):
        self.mark = len(self.lines)

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
        self.thread.join(timeout=2)
        lines = self.lines[self.mark:] if len(self.lines) > self.mark else self.lines
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# sources that define the batched DP kernel: its DRAM counters stay valid while these are unchanged
KERNEL_SOURCES = ("batch_kernel.cuh", "batch_score.cuh", "batch.h", "common.cuh", "engine.cuh")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2002_04561_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the DP kernel from the committed ncu summary,
    or None when the kernel sources changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "batch_dp_short_reads.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_launch")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cpu_baseline(batch, budget_s: float = 12.0):
    """Time the CPU oracle on a bounded prefix of the workload, all host cores."""
    import oracle
    sc = oracle.Scoring(*SCORING)
    threads = oracle.default_threads()
    # calibrate on a small prefix, then size the sample to about budget_s
    cal = batch.subset(np.arange(min(2000, batch.n_pairs)))
    t0 = time.perf_counter()
    oracle.score_batch(cal, sc, MODE, threads=threads)
    dt = time.perf_counter() - t0
    rate = cal.cells() / max(dt, 1e-6)
    n = int(min(batch.n_pairs, max(2000, batch.n_pairs * min(1.0, budget_s * rate / batch.cells()))))
    sub = batch.subset(np.arange(n))
    t0 = time.perf_counter()
    oracle.score_batch(sub, sc, MODE, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": sub.cells() / dt / 1e9, "unit": "GCUPS", "cores": threads, "kind": "oracle",
            "sample": f"first {n} of {batch.n_pairs} pairs ({sub.cells():.3e} cells), {dt:.1f} s"}


def oracle_sample(batch, sc_args, mode, want_cigar=False, budget_s: float = 3.0, matrix=None):
    """The CPU oracle on a bounded prefix of a secondary workload (all host
    cores over pairs), as GCUPS with the sample it ran."""
    import oracle
    sc = oracle.Scoring(*sc_args, matrix=matrix)
    threads = oracle.default_threads()
    fn = oracle.align_batch if want_cigar else oracle.score_batch
    n = 1
    while True:
        sub = batch.subset(np.arange(min(n, batch.n_pairs)))
        t0 = time.perf_counter()
        fn(sub, sc, mode, threads=threads)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or n >= batch.n_pairs:
            break
        n *= 4
    return {"GCUPS": sub.cells() / dt / 1e9, "cores": threads, "kind": "oracle",
            "sample": f"first {sub.n_pairs} of {batch.n_pairs} pairs ({sub.cells():.3e} cells), {dt:.2f} s"}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    batch = synth.short_reads()
    sc = oracle.Scoring(*SCORING)
    threads = oracle.default_threads()
    cal = batch.subset(np.arange(2000))
    t0 = time.perf_counter()
    oracle.score_batch(cal, sc, MODE, threads=threads)
    rate = cal.cells() / max(time.perf_counter() - t0, 1e-6)
    per_step_s = min(20.0, 150.0 / max(1, args.steps + args.warmup))
    n = int(min(batch.n_pairs, max(1000, per_step_s * rate / (batch.cells() / batch.n_pairs))))
    sub = batch.subset(np.arange(n))
    for _ in range(args.warmup):
        oracle.score_batch(sub, sc, MODE, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.score_batch(sub, sc, MODE, threads=threads)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sub.cells() * args.steps / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_pairs_sampled": n, "n_pairs_workload": batch.n_pairs},
        "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": threads, "kind": "oracle",
                         "sample": f"first {n} of {batch.n_pairs} pairs per step ({sub.cells():.3e} cells)"},
        "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def timed_events(fn, reps, stream):
    """Mean milliseconds of fn over reps runs, CUDA events on the stream, after one warm-up."""
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def serving_window_rates(sub, lat_ms):
    """Offered and achieved request rates over the middle 80 % of the requests:
    arrivals by submit time (s), completions (submit + latency) in completion
    order. A server that keeps up completes them over the same span as they
    arrive; one that falls behind spreads them over a longer one. The ends are
    left out (the start's empty queue, the last batch's drain)."""
    a = np.sort(np.asarray(sub, dtype=np.float64))
    c = np.sort(np.asarray(sub, dtype=np.float64) + np.asarray(lat_ms, dtype=np.float64) * 1e-3)
    lo, hi = int(0.1 * len(a)), int(0.9 * len(a)) - 1
    return (hi - lo) / (a[hi] - a[lo]), (hi - lo) / (c[hi] - c[lo])


def serving_workload(pkg, n_requests: int = 6000, loads=(0.5, 0.7, 0.9)):
    """The serving mix (70 % 100-300 bp, 25 % 1-10 kbp, 5 % 50-200 kbp, global
    affine +2/-3/-5/-2) through the native request queue: capacity with every
    request queued at once, then Poisson arrivals at each fraction of it;
    latency from submit to completion as the server measures it. A load counts
    as steady only where the achieved rate is at least 98 % of the offered one
    over the middle 80 % of the requests (the queue did not grow); the reported
    p50/p99 are those of the highest steady load."""
    import queue
    import threading
    sc = pkg.Scoring.make(2, -3, -5, -2)
    arr = synth.serving_mix(n_requests, rate_per_s=1.0)
    pairs = [arr.batch.pair(k) for k in range(n_requests)]
    cells = arr.batch.cells()

    def run(times):
        srv = pkg.Server(sc, mode=pkg.GLOBAL, max_wait_us=500, max_batch_pairs=8192)
        try:
            tq = queue.Queue()

            sub = np.zeros(n_requests)

            def submitter():
                t0 = time.perf_counter()
                for k in range(n_requests):
                    if times is not None:
                        delay = t0 + times[k] - time.perf_counter()
                        if delay > 0:
                            time.sleep(delay)
                    sub[k] = time.perf_counter()
                    tq.put(srv.submit(*pairs[k]))

            start = time.perf_counter()
            th = threading.Thread(target=submitter)
            th.start()
            lat = np.zeros(n_requests)
            for k in range(n_requests):
                _, lat[k] = srv.wait(tq.get())
            th.join()
            wall = time.perf_counter() - start
            return wall, lat * 1e-6, srv.stat("batches"), srv.stat("long_pairs"), sub

        finally:
            srv.close()

    run(None)  # warm-up: builds the context's scratch
    wall, _, _, _, _ = run(None)
    capacity = n_requests / wall
    res = {"requests": n_requests, "capacity_req_per_s": capacity,
           "capacity_GCUPS": cells / (n_requests / capacity) / 1e9, "loads": []}
    for load in loads:
        rate = load * capacity
        wall, lat, batches, longs, sub = run(arr.times / rate)
        offered_w, achieved_w = serving_window_rates(sub, lat)
        row = {"load": load, "offered_req_per_s": offered_w, "achieved_req_per_s": achieved_w,
               "achieved_over_offered": achieved_w / offered_w,
               "requests_over_wall_req_per_s": n_requests / wall,
               "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
               "batches": int(batches), "wavefront_pairs": int(longs)}
        for kind, name in enumerate(("short", "medium", "long")):
            sel = arr.kind == kind
            row[f"{name}_p50_ms"] = float(np.percentile(lat[sel], 50))
            row[f"{name}_p99_ms"] = float(np.percentile(lat[sel], 99))
        res["loads"].append(row)
    steady = [r for r in res["loads"] if r["achieved_over_offered"] >= 0.98]
    if steady:
        top = max(steady, key=lambda r: r["load"])
        res.update({"steady_load": top["load"], "p50_ms": top["p50_ms"], "p99_ms": top["p99_ms"],
                    "offered_req_per_s": top["offered_req_per_s"], "achieved_req_per_s": top["achieved_req_per_s"]})
    else:
        res["steady_load"] = None
    return res


def secondary_workloads(pkg, ctx, device):
    """The other workloads of the method, one line each (not the headline)."""
    import torch
    stream = torch.cuda.current_stream()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    out = {}
    # single 1,000 x 1,100 global pair with CIGAR (latency)
    b = synth.single_pair()
    sc = pkg.Scoring.make(2, -1, 0, -2)
    cig = torch.zeros(4096, dtype=torch.int32, device=device)
    res = torch.zeros(40, dtype=torch.uint8, device=device)
    args = (dev(b.q), dev(b.q_off), dev(b.s), dev(b.s_off))
    ms = timed_events(lambda: ctx.align_batch(*args, sc, pkg.GLOBAL, want=7, out=res, cigar=cig), 20, stream)
    out["single_pair_1000x1100_cigar"] = {"us": 1e3 * ms, "GCUPS": b.cells() / ms / 1e6,
                                          "cpu_oracle": oracle_sample(b, (2, -1, 0, -2), 0, want_cigar=True)}
    # the headline short reads with CIGAR (traceback DP, walk, compaction)
    b = synth.short_reads()
    sc = pkg.Scoring.make(*SCORING)
    args = (dev(b.q), dev(b.q_off), dev(b.s), dev(b.s_off))
    res = torch.zeros(b.n_pairs * 40, dtype=torch.uint8, device=device)
    cig = torch.zeros(int(b.q_len().sum() + b.s_len().sum() + b.n_pairs), dtype=torch.int32, device=device)
    ms = timed_events(lambda: ctx.align_batch(*args, sc, MODE, want=7, out=res, cigar=cig), 5, stream)
    dp = []
    for _ in range(3):
        ctx.align_batch(*args, sc, MODE, want=7, out=res, cigar=cig)
        dp.append(ctx.stat("dp_ms") + ctx.stat("dp32_ms"))
    out["short_reads_262144_semiglobal_cigar"] = {
        "ms": ms, "GCUPS": b.cells() / ms / 1e6, "dp_kernel_ms": statistics.median(dp),
        "cpu_oracle": oracle_sample(b, SCORING, MODE, want_cigar=True)}
    del res, cig
    # protein, local affine, score and CIGAR
    b = synth.protein_pairs()
    sc = pkg.Scoring.make(0, 0, -11, -1, matrix=synth.protein_matrix(3))
    args = (dev(b.q), dev(b.q_off), dev(b.s), dev(b.s_off))
    res = torch.zeros(b.n_pairs * 40, dtype=torch.uint8, device=device)
    ms = timed_events(lambda: ctx.align_batch(*args, sc, pkg.LOCAL, out=res), 5, stream)
    # the DP kernels alone (CUDA events around each launch, as for the headline kernel)
    kms = []
    for _ in range(5):
        ctx.align_batch(*args, sc, pkg.LOCAL, out=res)
        kms.append(ctx.stat("dp_ms") + ctx.stat("dp32_ms"))
    kernel_ms = statistics.median(kms)
    n_sm = torch.cuda.get_device_properties(device).multi_processor_count
    peak = n_sm * float(measured_peaks().get("sm_max_mhz", 2070.0)) * 1e6 * LANE_OPS_PER_CLK / I_ALG / 1e9
    cap = int(b.q_len().sum() + b.s_len().sum() + b.n_pairs)
    cig = torch.zeros(cap, dtype=torch.int32, device=device)
    ms2 = timed_events(lambda: ctx.align_batch(*args, sc, pkg.LOCAL, want=7, out=res, cigar=cig), 3, stream)
    out["protein_65536_local_affine"] = {"score_ms": ms, "score_GCUPS": b.cells() / ms / 1e6,
                                         "kernel_ms": kernel_ms, "kernel_GCUPS": b.cells() / kernel_ms / 1e6,
                                         "kernel_roofline_frac": b.cells() / kernel_ms / 1e6 / peak,
                                         "kernel": "batch_kernel<CellI16x2, LOCAL, shared-memory profile>",
                                         "cigar_ms": ms2, "cigar_GCUPS": b.cells() / ms2 / 1e6,
                                         "cpu_oracle": oracle_sample(b, (0, 0, -11, -1), 1,
                                                                     matrix=synth.protein_matrix(3))}
    # one long protein pair (titin-sized), local, 20 x 20 matrix: the wavefront's
    # matrix path, score + optimum cell, then start cell and CIGAR
    st = synth.Stream(3, 7)
    pq = synth.random_codes(st, 35_000, 20)
    ps, _ = synth.mutate(pq, np.array([0, len(pq)], np.int64), 0.3, 0.03, 0.5, 20, st)
    psc = pkg.Scoring.make(0, 0, -11, -1, matrix=synth.protein_matrix(3))
    dq, ds = dev(pq), dev(ps)
    pcig = torch.zeros(len(pq) + len(ps) + 4, dtype=torch.int32, device=device)
    ms = timed_events(lambda: ctx.align_long(dq, ds, psc, mode=pkg.LOCAL), 3, stream)
    ms2 = timed_events(lambda: ctx.align_long(dq, ds, psc, mode=pkg.LOCAL, want=pkg.WANT_SCORE | pkg.WANT_CIGAR,
                                              cigar=pcig), 2, stream)
    r, used = ctx.align_long(dq, ds, psc, mode=pkg.LOCAL, want=pkg.WANT_SCORE | pkg.WANT_CIGAR, cigar=pcig)
    cells = len(pq) * len(ps)
    small = synth.from_pairs([(pq[:8000], ps[:8000])], alphabet=20)
    out["long_protein_pair_35000_local_matrix"] = {
        "score_ms": ms, "score_GCUPS": cells / ms / 1e6, "cigar_total_ms": ms2, "cigar_words": int(used),
        "score": int(r["score"][0]),
        "cpu_oracle": oracle_sample(small, (0, 0, -11, -1), 1, matrix=synth.protein_matrix(3))}
    # 1 Mbp x 1 Mbp global affine: wavefront score, divide-and-conquer CIGAR
    b = synth.long_pair()
    qd, sd = dev(b.q), dev(b.s)
    sc = pkg.Scoring.make(2, -3, -5, -2)
    ms = timed_events(lambda: ctx.align_long(qd, sd, sc), 2, stream)
    hcig = np.zeros(len(b.q) + len(b.s) + 4, np.uint32)
    t0 = time.perf_counter()
    r, used = ctx.align_long(qd, sd, sc, want=7, cigar=hcig)
    hb_s = time.perf_counter() - t0
    # the oracle on a 20 kbp pair of the same generator (a 1 Mbp pair is 1e12 cells)
    peak32 = n_sm * float(measured_peaks().get("sm_max_mhz", 2070.0)) * 1e6 * LANE_OPS_PER_CLK / I_ALG32 / 1e9
    out["long_pair_1Mbp_global_affine"] = {"score_s": ms / 1e3, "score_GCUPS": b.cells() / ms / 1e6,
                                           "score_roofline_frac": b.cells() / ms / 1e6 / peak32,
                                           "roofline_peak_GCUPS": peak32,
                                           "cigar_total_s": hb_s, "cigar_words": int(used),
                                           "score": int(r["score"][0]),
                                           "cpu_oracle": oracle_sample(synth.long_pair(n=20_000, inversion=400),
                                                                       (2, -3, -5, -2), 0)}
    del qd, sd
    # learned band vs full DP on 65,536 pairs of 1-10 kbp (scores must be equal)
    train = synth.band_pairs(n_pairs=16384, seed=105)
    sc = pkg.Scoring.make(2, -3, -5, -2)
    t0 = time.perf_counter()
    loss = ctx.band_train(train.q, train.q_off, train.s, train.s_off, sc, epochs=60, lr=1e-3)
    train_s = time.perf_counter() - t0
    b = synth.band_pairs()
    args = (dev(b.q), dev(b.q_off), dev(b.s), dev(b.s_off))
    full = torch.zeros(b.n_pairs * 40, dtype=torch.uint8, device=device)
    band = torch.zeros(b.n_pairs * 40, dtype=torch.uint8, device=device)
    ms_full = timed_events(lambda: ctx.align_batch(*args, sc, pkg.GLOBAL, out=full), 2, stream)
    ms_band = timed_events(lambda: ctx.align_batch(*args, sc, pkg.GLOBAL, want=1 | pkg.BAND_LEARNED, out=band), 2,
                           stream)
    band_pass_cells = float(ctx.stat("band_cells"))  # cells of the last call's banded pass
    fr = full.cpu().numpy().view(pkg.RESULT_DTYPE)
    br = band.cpu().numpy().view(pkg.RESULT_DTYPE)
    accepted = int(((br["flags"] & pkg.FLAG_BAND_ACCEPTED) != 0).sum())
    fb = (br["flags"] & pkg.FLAG_FULL_FALLBACK) != 0
    fallback = int(fb.sum())
    fallback_cells = float((b.q_len().astype(np.float64) * b.s_len())[fb].sum())
    # the same route without the network: constant outputs (centre 0, one half-width
    # relative to the longer sequence)
    learned = ctx.band_model_get()
    const = {}
    ctx.set_option("band_margin_pct", 100)  # the fixed width as it is
    ctx.set_option("band_floor_pct", 0)
    for w in (0.1, 0.25, 0.4):
        p = np.zeros_like(learned)
        p[-1] = np.log(w)
        ctx.band_model_set(p)
        ms_c = timed_events(lambda: ctx.align_batch(*args, sc, pkg.GLOBAL, want=1 | pkg.BAND_LEARNED, out=band), 2,
                            stream)
        const[str(w)] = {"ms": ms_c, "scores_equal": bool(np.array_equal(
            fr["score"], band.cpu().numpy().view(pkg.RESULT_DTYPE)["score"]))}
    ctx.band_model_set(learned)
    ctx.set_option("band_margin_pct", 65)  # the shipped defaults again
    ctx.set_option("band_floor_pct", 30)
    best_const = min(const.values(), key=lambda v: v["ms"])["ms"]
    out["band_65536_1_10kbp_global_affine"] = {
        "pairs_per_s_full_dp": b.n_pairs / ms_full * 1e3, "pairs_per_s_learned_band": b.n_pairs / ms_band * 1e3,
        "speedup": ms_full / ms_band, "scores_equal": bool(np.array_equal(fr["score"], br["score"])),
        "band_accepted": accepted, "full_dp_fallback": fallback, "certified_share": accepted / b.n_pairs,
        "constant_band_ms": const, "speedup_over_best_constant_band": best_const / ms_band,
        "speedup_over_prior_constant_band": const["0.25"]["ms"] / ms_band,
        "full_dp_GCUPS": b.cells() / ms_full / 1e6,
        # the learned route as full-DP-equivalent cells per second, and as the cells it
        # relaxed (banded pass plus the fallback pairs' full DP) per second
        "learned_band_full_dp_equivalent_GCUPS": b.cells() / ms_band / 1e6,
        "learned_band_true_GCUPS": (band_pass_cells + fallback_cells) / ms_band / 1e6,
        "learned_band_cells": band_pass_cells + fallback_cells,
        "train_s": train_s, "train_loss": loss,
        "cpu_oracle_full_dp": oracle_sample(b, (2, -3, -5, -2), 0)}
    # serving: Poisson arrivals through the native request queue
    out["serving_mix_6000_global_affine"] = serving_workload(pkg)
    return out


def profile_long(n: int):
    """One global long pair of the long-pair generator's shape, scored twice by
    the wavefront (a small case for ncu captures of the wavefront kernel)."""
    import torch
    import paper_2002_04561_gb300 as pkg
    pkg.load(build_if_missing=True)
    ctx = pkg.Context(0)
    b = synth.long_pair(n=n, inversion=max(1, n // 50))
    q, s = torch.from_numpy(b.q).cuda(), torch.from_numpy(b.s).cuda()
    sc = pkg.Scoring.make(2, -3, -5, -2)
    for _ in range(2):
        r, _ = ctx.align_long(q, s, sc)
    torch.cuda.synchronize()
    print(json.dumps({"profile_long": n, "cells": b.cells(), "score": int(r["score"][0])}))


def profile_protein(n_pairs: int):
    """The protein workload's first n_pairs pairs (local affine, 20x20 matrix),
    score only, aligned twice (a small case for ncu captures of the batched
    kernel's shared-memory-profile variant)."""
    import torch
    import paper_2002_04561_gb300 as pkg
    pkg.load(build_if_missing=True)
    ctx = pkg.Context(0)
    ctx.set_option("profile", 1)
    b = synth.protein_pairs(n_pairs=n_pairs)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (dev(b.q), dev(b.q_off), dev(b.s), dev(b.s_off))
    sc = pkg.Scoring.make(0, 0, -11, -1, matrix=synth.protein_matrix(3))
    res = torch.zeros(b.n_pairs * 40, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        ctx.align_batch(*args, sc, pkg.LOCAL, out=res)
    torch.cuda.synchronize()
    print(json.dumps({"profile_protein": n_pairs, "cells": b.cells(), "dp_ms": ctx.stat("dp_ms"),
                      "dp32_ms": ctx.stat("dp32_ms"), "pairs16": ctx.stat("pairs16"), "pairs32": ctx.stat("pairs32")}))


def profile_cigar(n_pairs: int):
    """The first n_pairs short reads, semi-global, score + optimum cell + CIGAR,
    aligned twice (a small case for ncu captures of the traceback path)."""
    import torch
    import paper_2002_04561_gb300 as pkg
    pkg.load(build_if_missing=True)
    ctx = pkg.Context(0)
    ctx.set_option("profile", 1)
    b = synth.short_reads(n_pairs=n_pairs)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (dev(b.q), dev(b.q_off), dev(b.s), dev(b.s_off))
    sc = pkg.Scoring.make(*SCORING)
    res = torch.zeros(b.n_pairs * 40, dtype=torch.uint8, device="cuda")
    cig = torch.zeros(int(b.q_len().sum() + b.s_len().sum() + b.n_pairs), dtype=torch.int32, device="cuda")
    for _ in range(2):
        _, used = ctx.align_batch(*args, sc, MODE, want=7, out=res, cigar=cig)
    torch.cuda.synchronize()
    print(json.dumps({"profile_cigar": n_pairs, "cells": b.cells(), "dp_ms": ctx.stat("dp_ms"), "cigar_words": used}))


def profile_band(n_pairs: int):
    """The first n_pairs pairs of the band workload through the learned-band route
    with a constant network (half-width 0.4 x the longer sequence), twice (a case
    for ncu captures of the banded kernel)."""
    import torch
    import paper_2002_04561_gb300 as pkg
    pkg.load(build_if_missing=True)
    ctx = pkg.Context(0)
    b = synth.band_pairs(n_pairs=n_pairs)
    p = np.zeros(pkg.BAND_PARAMS, dtype=np.float32)
    p[-1] = np.log(0.4)
    ctx.band_model_set(p)
    ctx.set_option("band_margin_pct", 100)
    ctx.set_option("band_floor_pct", 0)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (dev(b.q), dev(b.q_off), dev(b.s), dev(b.s_off))
    sc = pkg.Scoring.make(2, -3, -5, -2)
    res = torch.zeros(b.n_pairs * 40, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        ctx.align_batch(*args, sc, pkg.GLOBAL, want=pkg.WANT_SCORE | pkg.BAND_LEARNED, out=res)
    torch.cuda.synchronize()
    print(json.dumps({"profile_band": n_pairs, "band_cells": ctx.stat("band_cells"),
                      "band_pass_ms": ctx.stat("band_pass_ms"), "accepted": ctx.stat("band_accepted")}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--pairs", type=int, default=262144, help="pairs per GPU (profiling runs use fewer)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-long", type=int, default=0, metavar="N",
                    help="profiling case: only the wavefront score of one N-letter long pair, twice")
    ap.add_argument("--profile-protein", type=int, default=0, metavar="N",
                    help="profiling case: only the protein local scores of the first N pairs, twice")
    ap.add_argument("--profile-cigar", type=int, default=0, metavar="N",
                    help="profiling case: only the first N short reads with CIGAR, twice")
    ap.add_argument("--profile-band", type=int, default=0, metavar="N",
                    help="profiling case: only the first N band pairs through the banded route, twice")
    args = ap.parse_args()
    ws, rank, local = dist_env()

    if args.profile_long:
        profile_long(args.profile_long)
        return
    if args.profile_protein:
        profile_protein(args.profile_protein)
        return
    if args.profile_cigar:
        profile_cigar(args.profile_cigar)
        return
    if args.profile_band:
        profile_band(args.profile_band)
        return

    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch
    import paper_2002_04561_gb300 as pkg
    assert torch.cuda.is_available(), "bench.py needs a CUDA GPU"
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    init_dist(ws, "nccl")
    pkg.load(build_if_missing=True)
    ctx = pkg.Context(local)
    ctx.set_option("profile", 1)

    # one global batch, this rank's share by the native partition (all pairs at N = 1)
    batch_all = synth.short_reads(n_pairs=args.pairs * ws, seed=2)
    mine = pkg.shard_plan(batch_all.q_off, batch_all.s_off, ws, rank)
    if ws == 1:
        batch = batch_all
    else:
        from paper_2002_04561_gb300.dist import take_pairs
        batch = synth.Batch(*take_pairs(batch_all.q, batch_all.q_off, mine),
                            *take_pairs(batch_all.s, batch_all.s_off, mine), batch_all.alphabet)
    cells = batch.cells()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    q, q_off, s, s_off = dev(batch.q), dev(batch.q_off), dev(batch.s), dev(batch.s_off)
    out = torch.zeros(batch.n_pairs * 40, dtype=torch.uint8, device=device)
    sc = pkg.Scoring.make(*SCORING)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=device)
    stream = torch.cuda.current_stream()

    def step():
        ctx.align_batch(q, q_off, s, s_off, sc, MODE, out=out)

    # the same batch as a graph plan (anyseq_plan_*): the whole launch sequence of
    # align_batch (packing, binning, both DP kernels, result records) replayed by one
    # graph launch per step, the letters checked after every run
    plan = pkg.Plan(batch.q_off, batch.s_off, sc, MODE, device=local)
    plan.q.copy_(q)
    plan.s.copy_(s)

    def plan_step():
        plan.run(stream)

    clocks = ClockSampler(local)
    clocks.start()  # running (first sample printed) before the warm-up
    for _ in range(max(3, args.warmup)):
        step()
        plan_step()
        plan.wait(stream)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    clocks.begin()
    # timed region: graph-plan steps (the headline value)
    step_ms, launches = [], 0
    per_call_launches = int(ctx.stat("launches"))
    for _ in range(args.steps):
        flush.fill_(1)  # evict L2 between timed steps (outside the events)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan_step()
        b.record(stream)
        plan.wait(stream)
        step_ms.append(a.elapsed_time(b))
        launches += per_call_launches
    # and align_batch steps: the per-call time, and CUDA events around the DP kernel
    call_ms, dp_ms = [], []
    for _ in range(args.steps):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        call_ms.append(a.elapsed_time(b))
        dp_ms.append(ctx.stat("dp_ms"))
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    total_ms = max_over_ranks(ws, sum(step_ms), device)
    call_total_ms = max_over_ranks(ws, sum(call_ms), device)
    all_cells = sum_over_ranks(ws, float(cells) * args.steps, device)
    value = all_cells / (total_ms / 1e3) / 1e9
    call_value = all_cells / (call_total_ms / 1e3) / 1e9

    # end to end through the C ABI with pinned host buffers: (1) one anyseq_align_batch
    # call per step from host buffers; (2) the graph plans of a stream of batches: two
    # plans of the shape on two streams, each step uploading its letters from pinned
    # host memory, replaying the graph and downloading its result records
    # (anyseq_plan_upload / _run / _download / _wait), so that one step's copies
    # overlap the other plan's run. Every copy is inside the timed region.
    hq, hqo = torch.from_numpy(batch.q).pin_memory(), torch.from_numpy(batch.q_off).pin_memory()
    hs, hso = torch.from_numpy(batch.s).pin_memory(), torch.from_numpy(batch.s_off).pin_memory()
    hout = torch.zeros(batch.n_pairs * 40, dtype=torch.uint8).pin_memory()
    ctx.align_batch(hq, hqo, hs, hso, sc, MODE, out=hout)
    e2e_ms = []
    barrier(ws)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ctx.align_batch(hq, hqo, hs, hso, sc, MODE, out=hout)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    call_e2e_total = max_over_ranks(ws, sum(e2e_ms), device)
    call_e2e_value = all_cells / (call_e2e_total / 1e3) / 1e9
    plan2 = pkg.Plan(batch.q_off, batch.s_off, sc, MODE, device=local)
    plans, pstreams = [plan, plan2], [torch.cuda.Stream(device), torch.cuda.Stream(device)]
    pouts = [torch.zeros(batch.n_pairs * 40, dtype=torch.uint8).pin_memory() for _ in range(2)]
    for i in range(2):  # capture both graphs
        plans[i].upload(hq, hs, pstreams[i])
        plans[i].run(pstreams[i])
        plans[i].download(pouts[i], pstreams[i])
        plans[i].wait(pstreams[i])
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for k in range(args.steps):
        i = k & 1
        if k >= 2:
            plans[i].wait(pstreams[i])  # step k - 2 on this plan: done, letters checked
        plans[i].upload(hq, hs, pstreams[i])
        plans[i].run(pstreams[i])
        plans[i].download(pouts[i], pstreams[i])
    for i in range(2):
        plans[i].wait(pstreams[i])
    e2e_total = max_over_ranks(ws, 1e3 * (time.perf_counter() - t0), device)
    e2e_value = all_cells / (e2e_total / 1e3) / 1e9
    assert np.array_equal(pouts[0].numpy().view(pkg.RESULT_DTYPE)["score"], hout.numpy().view(pkg.RESULT_DTYPE)["score"])
    plan2.close()
    h2d = batch.q.nbytes + batch.s.nbytes
    d2h = hout.numel()

    # the host-buffer and device-buffer calls must give the same results (untimed)
    res = out.cpu().numpy().view(pkg.RESULT_DTYPE)
    hres = hout.numpy().view(pkg.RESULT_DTYPE)
    pres = plan.results()
    assert np.array_equal(res["score"], hres["score"])
    assert np.array_equal(res["score"], pres["score"]) and np.array_equal(res["end_s"], pres["end_s"])
    plan.close()

    gathered = None
    if ws > 1:
        # the one exchange of the path: every record to rank 0, in the global batch's order
        from paper_2002_04561_gb300 import dist as pdist
        recs = pdist.align_batch_sharded(ctx, batch_all.q, batch_all.q_off, batch_all.s, batch_all.s_off, sc, MODE)
        if rank == 0:
            assert len(recs) == batch_all.n_pairs
            assert np.array_equal(recs["score"][mine], hres["score"])
            gathered = int(len(recs))

    peaks = measured_peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_gcups = n_sm * f_max * LANE_OPS_PER_CLK / I_ALG / 1e9
    dp_avg = statistics.mean(dp_ms)
    achieved = cells / (dp_avg / 1e3) / 1e9
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_gcups, "unit": "GCUPS",
            "frac": achieved / peak_gcups, "traffic": profiled_traffic(),
            "peak_basis": f"{n_sm} SMs x {f_max / 1e6:.0f} MHz (max) x I_SM {LANE_OPS_PER_CLK:.0f} lane-ops/clk / "
                          f"I_alg {I_ALG} ops per cell; I_SM = 6 ops / max(4/{HALF_RATE}, 2/{FULL_RATE}, "
                          f"6/{ISSUE_RATE}) clk for the cell's 4 half-rate + 2 full-rate ops per lane-word",
            "kernel": "batch_kernel<CellI16x2, SEMIGLOBAL>", "kernel_ms": dp_avg,
            "frac_nominal_128": achieved / (peak_gcups * NOMINAL_LANE_OPS / LANE_OPS_PER_CLK)}
    if clk.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / (n_sm * clk["sm_mhz"] * 1e6 * LANE_OPS_PER_CLK / I_ALG / 1e9)

    line = {
        "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int16x2", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.pairs == 262144 else f"short_reads_{args.pairs}_semiglobal_affine",
                   "n_pairs_per_gpu": batch.n_pairs, "cells_per_gpu": cells,
                   "query_len": "100-250", "target": "query + 4% sub + 1% indel + 20bp flanks",
                   "scoring": "semiglobal +1/-4 open -6 extend -1", "l2": "flushed between steps (258 MB write)",
                   "pairs_per_s": batch.n_pairs * ws * args.steps / (total_ms / 1e3),
                   "parallelism": f"dp{ws}",
                   "partition": "one global batch, length-balanced round-robin of cell-count bins per rank",
                   "gathered_pairs": gathered,
                   "step": "one graph-plan replay of the batched path (anyseq_plan_run) and its letter check "
                           "(anyseq_plan_wait); kernel time for the roofline from events around the DP kernel "
                           "in anyseq_align_batch steps over the same batch",
                   "align_batch_ms_per_step": call_total_ms / args.steps,
                   "align_batch_GCUPS": call_value},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": "GCUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "two graph plans on two streams: per step anyseq_plan_upload of the letters from pinned "
                        "host memory, anyseq_plan_run, anyseq_plan_download of the records, anyseq_plan_wait "
                        "before the plan's next step; one step's copies overlap the other plan's run",
                "align_batch_per_call": {"value": call_e2e_value, "unit": "GCUPS",
                                         "h2d_bytes_per_step": h2d + batch.q_off.nbytes + batch.s_off.nbytes,
                                         "d2h_bytes_per_step": d2h}},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(batch)
    if rank == 0 and not args.no_extra:
        del q, q_off, s, s_off, out
        torch.cuda.empty_cache()
        line["workloads"] = secondary_workloads(pkg, ctx, device)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
