#!/usr/bin/env python
"""Benchmark of MTGP generation on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c2|c1|c3|c4]

A step is one pass of the whole generation path over one batch: for the
default workload (C2) every one of 128 MTGP11213 parameter sets produces 2^24
numbers in each of uint32, float [1,2) and float [0,1) -- 384 generator
instances, one thread block each, in one launch (about 24 GiB written).  The
step continues every generator's stream, so successive steps do new work.

Prints one JSON line (rank 0).  Under torchrun each rank runs its own shard
(distinct generator IDs, same sizes: weak scaling, no collective on the data
path); the time is the max over ranks.  `--impl reference` times the CPU oracle
on the host cores instead (rank 0 only).
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

METRIC = "MTGP Gnum/s & HBM write GB/s vs peak (plain vs batched); served p50/p99 latency"
KERNEL_SOURCES = ["paper_1005_4973_gb300/csrc/mtgp_device.cuh", "paper_1005_4973_gb300/csrc/mtgp_pairs.cuh",
                  "paper_1005_4973_gb300/csrc/mtgp_layout.h"]
# generation kernel of each launch form (mtgp_config.form)
FORM_KERNEL = {0: "k_generate", 1: "k_split", 2: "k_flow", 3: "k_wide", 4: "k_pairs", 5: "k_dual"}
DTYPE = "u32+f32"       # integer recursion; f32 outputs by mantissa fill (one exact subtraction for [0,1))


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


WORKLOAD_DESC = {
    "c1": "C1: MTGP11213 x 1 generator x 2^20 u32",
    "c2": "C2: MTGP11213, 128 sets x 2^24 x {u32, f[1,2), f[0,1)}, blocked",
    "c3": "C3: MTGP23209 + MTGP44497, 128 sets each x 2^26 f[0,1)",
    "c4": "C4: 8192 generators, mixed mexp, log-uniform 2^10..2^24, persistent",
    "c2s": "C2 at 2^20 numbers per generator (profiling size)",
    "c2m": "C2 at 2^22 numbers per generator (profiling size, split into pieces)",
    "c3s": "C3 at 2^22 numbers per generator (profiling size, split into pieces)",
    "paper": "Sec. 4.4: 5e7 f[0,1) numbers from 108 MTGP11213 generators",
}


def workload(name: str, rank: int):
    from paper_1005_4973_gb300 import workloads as WL
    wl = {"c1": WL.c1, "c2": WL.c2, "c3": WL.c3, "c4": WL.c4,
          "c2s": lambda: WL.c2(n=1 << 20),
          "c2m": lambda: WL.c2(n=1 << 22),
          "c3s": lambda: WL.c3(n=1 << 22),
          "paper": lambda: WL.paper()}[name]()
    if rank:
        for g in wl.gens:                  # distinct streams per rank
            g.gen_id += rank * 1_000_000
            g.seed += rank
    return wl


def max_over_ranks(torch, dist, x: float, device) -> float:
    """The slowest rank's value (whole-job time is the max over ranks)."""
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.samples, self.proc, self.marks = [], None, []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(device_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.samples.append((time.perf_counter(), parts))

    def mark(self):
        self.marks.append(time.perf_counter())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [p for t, p in self.samples if t0 <= t <= t1]
        window = "timed region"
        if len(rows) < 3:                   # short region: widen to the loaded run around it
            rows = [p for t, p in self.samples if self.marks and self.marks[0] <= t <= t1]
            window = "warm-up and timed region"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(rows[0][1]),
                "power_w_max": max((num(r[2]) or 0.0) for r in rows), "reasons": reasons,
                "samples": len(rows), "window": window}


def cpu_baseline(wl, numbers_per_gen: int, batch: int = 32):
    """The oracle, as it stands, on the host cores over a bounded sample."""
    import oracle as O
    O.build()
    threads = os.cpu_count() or 1
    specs = wl.gens
    dts = {r[0]: r[1] for r in wl.requests}
    t0 = time.perf_counter()
    done = 0
    for b in range(0, len(specs), batch):
        ps, sts = [], []
        for g in specs[b:b + batch]:
            p = O.params_draw(g.mexp, g.param_seed, g.id)
            ps.append(p)
            sts.append(O.seed_state(p, g.gen_id, g.seed))
        O.generate_many(ps, sts, [numbers_per_gen] * len(ps), [dts[b + i] for i in range(len(ps))], threads)
        done += numbers_per_gen * len(ps)
    dt = time.perf_counter() - t0
    return done / dt / 1e9, threads, dt, done


def run_reference(args, rank, world):
    """`--impl reference`: the CPU oracle timed on the host cores (rank 0)."""
    if rank != 0:
        return
    import oracle as O
    O.build()
    wl = workload(args.workload, 0)
    per_step = args.ref_numbers
    threads = os.cpu_count() or 1
    ps, sts, dts = [], [], []
    for r in wl.requests:
        g = wl.gens[r[0]]
        p = O.params_draw(g.mexp, g.param_seed, g.id)
        ps.append(p)
        sts.append(O.seed_state(p, g.gen_id, g.seed))
        dts.append(r[1])

    def step():
        O.generate_many(ps, sts, [per_step] * len(ps), dts, threads)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    nums = per_step * len(ps) * args.steps
    value = nums / dt / 1e9
    sample = f"{len(ps)} generator instances of {wl.name} x {per_step} numbers per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gnum/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE,
        "data": "synthetic", "config": {"workload": WORKLOAD_DESC[args.workload], "generators": len(ps)},
        "cpu_baseline": {"value": value, "unit": "Gnum/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Gnum/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_batched(torch, M, sample: int = 512):
    """C4: 8192 generators in one graph-captured persistent launch (timed over
    replays), against one plain single-generator launch per generator on the
    first `sample` generators (same streams, timed separately)."""
    from paper_1005_4973_gb300 import workloads as WL
    wl = WL.c4()
    ps = [M.mtgp_params_draw(g.mexp, g.param_seed, g.id) for g in wl.gens]
    pool = M.Pool(ps, [g.gen_id for g in wl.gens], [g.seed for g in wl.gens])
    total = wl.total_numbers
    out = torch.empty(total, dtype=torch.int32, device="cuda")
    # the project's autotuner picks form, block size, words per round,
    # persistence, pieces and layout (C4's lengths differ: blocked only); it
    # restores every state, and the graph captures the chosen configuration
    t0 = time.perf_counter()
    best, tune_ms, layout = pool.autotune(wl.requests, out)
    tune_s = time.perf_counter() - t0
    # room for the jump-ahead pieces of the long generators (the plan splits
    # about 16 work items' worth per SM)
    graph = M.Graph(pool, max_items=2 * len(wl.gens))
    graph.set_requests(wl.requests, out)
    for _ in range(3):                                       # warm-up replays
        graph.launch()
    steps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        graph.launch()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    assert graph.errors() == 0
    graph.close()
    # one plain launch per generator (a one-request call each, no jump-ahead
    # pieces), first `sample` generators
    pool.set_config(threads=128, persistent=0, pieces=1)
    sub = wl.requests[:sample]
    n_sub = sum(r[2] for r in sub)
    for r in sub[:8]:
        pool.generate([r], out)
    torch.cuda.synchronize()
    e0.record()
    for r in sub:
        pool.generate([r], out)
    e1.record()
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    pool.close()
    return {"workload": "C4: 8192 generators, mexp uniform over {11213, 23209, 44497}, lengths "
                        "floor(2^U(10,24)), u32/f[0,1) alternating, blocked",
            "value": total / (ms * 1e-3) / 1e9, "unit": "Gnum/s", "ms_per_launch": ms,
            "hbm_write_gbs": 4 * total / (ms * 1e-3) / 1e9, "numbers": total,
            "form": "one graph-captured launch: jump-ahead piece states, then the persistent generation "
                    "launch (longest first), in the configuration the autotuner chose",
            "autotuned": {"config": best.as_dict(), "layout": ["blocked", "interleaved"][layout],
                          "tuned_call_ms": tune_ms, "tuning_s": tune_s},
            "plain_per_generator": {"value": n_sub / (ms_plain * 1e-3) / 1e9, "unit": "Gnum/s",
                                    "generators": len(sub), "launches": len(sub),
                                    "note": "one launch per generator, first %d generators of C4" % len(sub)}}


def run_c1(torch, M, reps: int = 50):
    """C1: one MTGP11213 generator, 2^20 u32 per call (a latency figure: one
    stream, split into jump-ahead pieces by the default configuration);
    median CUDA-event time of `reps` calls after warm-up."""
    from paper_1005_4973_gb300 import workloads as WL
    wl = WL.c1()
    g = wl.gens[0]
    pool = M.Pool([M.mtgp_params_draw(g.mexp, g.param_seed, g.id)], [g.gen_id], [g.seed])
    out = torch.empty(wl.total_numbers, dtype=torch.int32, device="cuda")
    for _ in range(5):
        pool.generate(wl.requests, out)
    ms = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(reps):
        e0.record()
        pool.generate(wl.requests, out)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    pool.close()
    med = statistics.median(ms)
    return {"workload": "C1: MTGP11213, one generator, 2^20 u32 per call", "ms_median": med,
            "ms_min": min(ms), "value": wl.total_numbers / (med * 1e-3) / 1e9, "unit": "Gnum/s",
            "calls": reps, "note": "latency of one call (host planning and the jump-ahead kernel included)"}


def run_c3(torch, M, peak: float, steps: int = 5):
    """C3: 128 parameter sets of MTGP23209 and of MTGP44497, 2^26 f[0,1)
    each, one mexp at a time (32 GiB of output each); per mexp the step's
    Gnum/s and the generation launch's roofline (CUDA events recorded by the
    pool around it)."""
    from paper_1005_4973_gb300 import workloads as WL
    res = {}
    for mexp in (23209, 44497):
        wl = WL.c3(mexps=(mexp,))
        ps = [M.mtgp_params_draw(g.mexp, g.param_seed, g.id) for g in wl.gens]
        pool = M.Pool(ps, [g.gen_id for g in wl.gens], [g.seed for g in wl.gens])
        total = wl.total_numbers
        out = torch.empty(total, dtype=torch.int32, device="cuda")
        for _ in range(3):
            pool.generate(wl.requests, out)
        pool.set_timing(steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            pool.generate(wl.requests, out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        jump_ms, gen_ms = pool.kernel_times(steps)
        cfg = pool.config.as_dict()
        pool.close()
        del out
        torch.cuda.empty_cache()
        alg = 4 * total + sum(8 * p.N for p in ps)
        ach = alg / (statistics.mean(gen_ms) * 1e-3) / 1e9
        res[f"mexp{mexp}"] = {"value": total / (ms * 1e-3) / 1e9, "unit": "Gnum/s", "ms_per_step": ms,
                              "numbers": total, "steps": steps, "launch": cfg,
                              "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                           "frac": ach / peak, "avg_launch_ms": statistics.mean(gen_ms),
                                           "avg_jump_ms": statistics.mean(jump_ms)}}
    return res


# Sec. 4.4, Table 2: milliseconds for 5e7 numbers from 108 MTGP11213
# generators on the GTX 260 and GT 120 (u32, f[1,2), f[0,1)).
PAPER_MS = {"GTX 260": (4.7, 4.8, 5.0), "GT 120": (38.2, 38.9, 39.8)}


def run_paper(torch, M, reps: int = 20):
    """Sec. 4.4's workload: 5e7 numbers of each dtype from 108 MTGP11213
    generators, default launch configuration; median CUDA-event time of
    `reps` calls after warm-up."""
    from paper_1005_4973_gb300 import workloads as WL
    res = []
    for dt, name in ((0, "u32"), (1, "f[1,2)"), (2, "f[0,1)")):
        wl = WL.paper(dtype=dt)
        ps = [M.mtgp_params_draw(g.mexp, g.param_seed, g.id) for g in wl.gens]
        pool = M.Pool(ps, [g.gen_id for g in wl.gens], [g.seed for g in wl.gens])
        out = torch.empty(wl.total_numbers, dtype=torch.int32, device="cuda")
        for _ in range(3):
            pool.generate(wl.requests, out)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            pool.generate(wl.requests, out)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        res.append({"dtype": name, "ms": ms, "gnums": wl.total_numbers / ms / 1e6,
                    "paper_ms": {k: v[dt] for k, v in PAPER_MS.items()}})
        pool.close()
        del out
    return {"workload": "Sec. 4.4: 5e7 numbers from 108 MTGP11213 generators per dtype, blocked",
            "timing": "median of %d calls, CUDA events around the call (host planning included)" % reps,
            "runs": res}


# Output arena of the served run.  A request holds 4 n bytes from admission
# until it completes, about ceil(n / chunk) ticks later, so by Little's law the
# arena must hold arrival rate x E[4 n ceil(n / chunk)] x tick time: about
# 53 GB at 0.8 of a 725 Gnum/s batched rate with chunk 2^22 and 3 ms ticks.
# 96 GiB leaves headroom; 24 GiB capped the sustained rate near 190 Gnum/s.
SERVE_ARENA = 96 << 30
# Numbers per request per tick: 2^21 halves the typical wait for a tick
# against 2^22 at the same p99 (measured at 0.5 load: p50 4.6 vs 8.9 ms).
SERVE_CHUNK = 1 << 21
# block size of the served launches: 128 measured best at high load (0.8 of the batched rate:
# 624 against 553 Gnum/s sustained, p99 89 against 148 ms); 256 is 7 % better at 0.5
SERVE_THREADS = 128


def run_served(torch, M, batched_gnums: float, fracs=(0.25, 0.5, 0.8), requests: int = 50000,
               warm: int = 2000):
    """C5: Poisson arrivals over 65536 resident generators at fractions of the
    measured batched rate, run by the library's native request loop; p50/p99
    latency (device completion minus host submission) over `requests` requests
    after `warm` warm-up arrivals."""
    import numpy as np
    from paper_1005_4973_gb300 import workloads as WL
    gens = WL.c5_pool()
    ps = [M.mtgp_params_draw(g.mexp, g.param_seed, g.id) for g in gens]
    pool = M.Pool(ps, [g.gen_id for g in gens], [g.seed for g in gens])
    pool.set_config(threads=SERVE_THREADS)
    mean_len = WL.expected_log_uniform_len(8.0, 26.0)
    results = []
    for frac in fracs:
        rate = frac * batched_gnums * 1e9 / mean_len
        arrivals = WL.c5_arrivals(rate, warm + requests, pool_size=len(gens), seed=13 + int(100 * frac))
        srv = M.Server(pool, arena_bytes=SERVE_ARENA, chunk=SERVE_CHUNK, max_active=4096)
        lat, done = srv.run_trace(arrivals)
        st = srv.stats()
        srv.close()
        arr = np.array([a[0] for a in arrivals[warm:]])
        n = np.array([a[3] for a in arrivals[warm:]], dtype=np.float64)
        lat_ms = lat[warm:] * 1e3
        span = float(done[warm:].max() - arr.min())
        results.append({"rate_frac": frac, "rate_req_s": rate, "requests": requests, "warmup_requests": warm,
                        "offered_gnums": float(n.sum() / (arr.max() - arr.min()) / 1e9),
                        "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                        "mean_ms": float(lat_ms.mean()),
                        "sustained_gnums": float(n.sum() / span / 1e9) if span > 0 else None,
                        "ticks": int(st["ticks"])})
    pool.close()
    return {"workload": "C5: 65536 resident generators (mexp mix as C4), Poisson arrivals, lengths "
                        "floor(2^U(8,26)), u32/f[0,1) 50/50, continuous batching",
            "mean_len": mean_len, "chunk": SERVE_CHUNK, "max_active": 4096, "arena_bytes": SERVE_ARENA,
            "threads": SERVE_THREADS,
            "latency": "device completion event minus host submission", "loop": "mtgp_server_run_trace (native)",
            "rates": results}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c2s", "c2m", "c3s", "paper"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-numbers", type=int, default=1 << 24, help="numbers per generator in the CPU sample")
    ap.add_argument("--ref-numbers", type=int, default=1 << 20, help="numbers per generator per reference step")
    ap.add_argument("--config", default="", help="JSON launch config overrides (threads, form, persistent, ...)")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched (C4) and served (C5) measurements")
    ap.add_argument("--serve-requests", type=int, default=50000, help="C5 requests timed per arrival rate")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_1005_4973_gb300 as M
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    wl = workload(args.workload, rank)
    ps = [M.mtgp_params_draw(g.mexp, g.param_seed, g.id) for g in wl.gens]
    pool = M.Pool(ps, [g.gen_id for g in wl.gens], [g.seed for g in wl.gens])
    if args.workload in ("c3", "c3s", "c4"):
        pool.set_config(persistent=1)
    if args.config:
        pool.set_config(**json.loads(args.config))
    cfg = pool.config.as_dict()
    total = wl.total_numbers
    out = torch.empty(total, dtype=torch.int32, device="cuda")
    reqs = wl.requests
    stream = torch.cuda.current_stream()

    # write-only roofline probe on the same buffer
    probe_words = (min(total, 1 << 31) // 4) * 4
    for _ in range(3):
        M.mtgp_fill_probe(out, probe_words)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    for _ in range(5):
        M.mtgp_fill_probe(out, probe_words)
    pe1.record(stream)
    torch.cuda.synchronize()
    write_probe_gbs = 5 * 4 * probe_words / (pe0.elapsed_time(pe1) * 1e-3) / 1e9

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_id = vis.split(",")[local].strip() if vis else str(local)
    sampler = ClockSampler(smi_id) if rank == 0 else None
    if sampler:
        time.sleep(0.3)
        sampler.mark()
    for _ in range(args.warmup):
        pool.generate(reqs, out)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    pool.set_timing(args.steps)                          # events around each call's two launches
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    launches0 = pool.launch_count()
    t_host0 = time.perf_counter()
    e0.record(stream)
    for k in range(args.steps):
        starts[k].record(stream)
        pool.generate(reqs, out)
        ends[k].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_host1 = time.perf_counter()
    launches = pool.launch_count() - launches0
    jump_ms, gen_ms = pool.kernel_times(args.steps)
    pool.set_timing(0)
    errs = pool.errors()                                 # shape / bounded-wait flags of the timed launches
    if errs:
        raise SystemExit(f"bench: kernel error flags {errs:#x} set during the timed steps; outputs invalid")
    if dist:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    launch_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    if dist:
        ms_total = max_over_ranks(torch, dist, ms_total, "cuda")
    clocks = sampler.summary(t_host0, t_host1) if sampler else None

    numbers_all = total * args.steps * world
    value = numbers_all / (ms_total * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    state_bytes = sum(8 * p.N for p in ps)
    alg_bytes = 4 * total + state_bytes                  # per launch: outputs + state load/store
    avg_launch = statistics.mean(launch_ms)              # whole step (jump + generation)
    avg_gen = statistics.mean(gen_ms)                    # the generation launch alone
    avg_jump = statistics.mean(jump_ms)
    achieved = alg_bytes / (avg_gen * 1e-3) / 1e9
    kname = FORM_KERNEL.get(cfg["form"], "k_generate")
    traffic, traffic_src = None, None                    # ncu DRAM bytes, scaled to this launch
    summary = os.path.join(ROOT, "profiles", f"{kname}_traffic.json")
    if os.path.exists(summary) and args.workload in ("c2", "c2s", "c2m"):
        with open(summary) as f:
            tj = json.load(f)
        if tj.get("kernel_hash") == kernel_hash():
            traffic = float(tj["traffic_bytes_per_number"]) * total
            traffic_src = os.path.relpath(summary, ROOT)

    e2e = None
    if not args.no_e2e and rank == 0:
        host = torch.empty(total, dtype=torch.int32, pin_memory=True)
        # warm-up as for the device-timed steps (at least 3): allocates the
        # staging buffers; the first passes into a fresh pinned buffer are slower
        for _ in range(max(args.warmup, 3)):
            pool.generate_host(reqs, host)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            pool.generate_host(reqs, host)
        dt = time.perf_counter() - t0
        # the host link on this machine: device-to-host copies of the same bytes into the same pinned
        # buffer, in two halves on two streams (two copy engines), best of three -- the ceiling
        # the end-to-end figure runs against
        dev = torch.empty(total, dtype=torch.int32, device="cuda")
        half = total // 2
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        link_gbs = 0.0
        for _ in range(3):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            for k, st in enumerate(streams):
                with torch.cuda.stream(st):
                    sl = slice(0, half) if k == 0 else slice(half, total)
                    host[sl].copy_(dev[sl], non_blocking=True)
            torch.cuda.synchronize()
            link_gbs = max(link_gbs, 4 * total / (time.perf_counter() - t1) / 1e9)
        del dev
        e2e = {"value": total * args.e2e_steps / dt / 1e9, "unit": "Gnum/s",
               "h2d_bytes_per_step": 64 * len(reqs), "d2h_bytes_per_step": 4 * total,
               "steps": args.e2e_steps, "warmup": max(args.warmup, 3),
               "path": "mtgp_pool_generate_host into pinned host memory",
               "link_probe_gbs": link_gbs,
               "frac_of_link": 4 * total * args.e2e_steps / dt / 1e9 / link_gbs}
        del host

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        v, cores, dt, done = cpu_baseline(wl, args.cpu_numbers)
        cpu = {"value": v, "unit": "Gnum/s", "cores": cores, "kind": "oracle",
               "sample": f"all {len(wl.gens)} generator instances of {wl.name} x {args.cpu_numbers} numbers "
                         f"({done:.3g} numbers, {dt:.1f} s)"}

    extras = {}
    if not args.no_extras and rank == 0 and world == 1 and args.workload == "c2":
        del out
        torch.cuda.empty_cache()
        extras["paper_workload"] = run_paper(torch, M)
        torch.cuda.empty_cache()
        extras["c1"] = run_c1(torch, M)
        torch.cuda.empty_cache()
        extras["c3"] = run_c3(torch, M, peak)
        torch.cuda.empty_cache()
        extras["batched"] = run_batched(torch, M)
        torch.cuda.empty_cache()
        extras["served"] = run_served(torch, M, extras["batched"]["value"], requests=args.serve_requests)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gnum/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE, "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC[args.workload],
                       "generators": len(wl.gens), "numbers_per_step": total,
                       "bytes_written_per_step": 4 * total,
                       "l2": "outputs larger than the 129 MB L2 every step; no flush",
                       "launch": cfg, "parallelism": f"generator shards x{world}"},
            "hbm_write_gbs": 4 * numbers_all / world / (ms_total * 1e-3) / 1e9,
            "write_probe_gbs": write_probe_gbs,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
                         "peak_kind": peak_kind, "kernel": kname, "alg_bytes_per_launch": alg_bytes,
                         "avg_launch_ms": avg_gen, "timing": "CUDA events around the generation launch, "
                         "recorded by the pool on the launching stream in every timed step",
                         "frac_of_write_probe": achieved / write_probe_gbs},
            "step_roofline": {"achieved": alg_bytes / (avg_launch * 1e-3) / 1e9, "avg_step_ms": avg_launch,
                              "avg_jump_ms": avg_jump, "frac": alg_bytes / (avg_launch * 1e-3) / 1e9 / peak},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "kernel_hash": kernel_hash(),
        }
        line.update(extras)
        print(json.dumps(line))
    if sampler:
        sampler.stop()
    pool.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
