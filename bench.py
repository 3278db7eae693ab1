"""Benchmark of the ASSE hot path on GB300: one step = ingest one slice of
(aip, bip) pairs into the AT pool + close the slice (scan with the fused
refresh, restore, estimate) + read the report on the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload link]
    python bench.py --impl reference ...    # the CPU oracle on the same workload

Prints one JSON line (rank 0).  With N > 1 (torchrun, one process per GPU)
every rank runs an independent replica of the workload (the method has no
data exchange between pools): weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "pkts/s AT ingest+SP estimate per slice, p99 slice latency, % of sector roofline"
N_SLICES_CYCLED = 8
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
# learned estimator: 68 used features -> 256 -> 256 -> 1 (multiply-adds x 2)
MLP_FLOP_PER_ROW = 2 * (68 * 256 + 256 * 256 + 256)
# dram__bytes_read.sum + dram__bytes_write.sum of one launch, from an ncu
# capture of the kernel, keyed by (workload, counter, kernel): the bytes and
# the id of the kernel source they were taken from (kernel_source_id below).
# A figure whose source id no longer matches the current sources is reported
# as null (the kernel has changed since the capture).
TRAFFIC = {
    ("long", "hist", "ingest"): (1295601920, "d0191276ba84"),
    ("long", "hist", "hist_scan"): (147243248, "bd35d6abdfed"),
    ("link", "at", "ingest"): (201379072, "d0191276ba84"),
    ("link", "at", "scan"): (96883456, "7fe98d3eebca"),
    ("long", "at", "scan"): (1081540752, "7fe98d3eebca"),
}
KERNEL_SOURCES = {
    "ingest": ["asse_ingest.cu", "asse_device.cuh", "asse_internal.h"],
    "scan": ["asse_scan.cu", "asse_swar.cuh", "asse_bytes.h", "asse_device.cuh", "asse_internal.h", "asse_ptx.cuh"],
    "hist_scan": ["asse_hist.cu", "asse_swar.cuh", "asse_bytes.h", "asse_device.cuh", "asse_internal.h"],
}


def kernel_source_id(kernel: str) -> str:
    """First 12 hex digits of the SHA-256 of the kernel's source files, with
    line comments and blank lines left out (a comment does not change what
    the kernel does)."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1807_01527_gb300", "csrc", name), encoding="utf-8") as f:
            for line in f:
                code = line.split("//", 1)[0].strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:12]


def traffic_of(workload: str, counter: str, kernel: str):
    """(bytes per launch or None, capture id or None, whether it is current)."""
    t = TRAFFIC.get((workload, counter, kernel))
    if t is None:
        return None, None, False
    current = t[1] == kernel_source_id(kernel)
    return (t[0] if current else None), t[1], current


def workload_desc(w) -> dict:
    return {"workload": "%s: k=%d, %d pairs/slice, %d hosts Zipf(%.1f), theta=%d, pool r=%d x %d ATVs x g=%d ATs"
                        % (w.name, w.k, w.n_per_slice, w.n_hosts, w.zipf, w.theta, w.r, 1 << w.E_log2, w.g),
            "k": w.k, "pairs_per_slice": w.n_per_slice, "theta": w.theta, "r": w.r, "atvs_per_row": 1 << w.E_log2,
            "g": w.g, "c": w.c, "u": w.u, "s": w.s, "seed": w.seed}


def peaks(kind: str = "hbm_gbs"):
    """Measured peak (HBM GB/s, or BF16 TFLOP/s burst / sustained) and its source."""
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return float(p[kind]), "of measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "bf16_tflops": FALLBACK_BF16_TFLOPS,
                "bf16_tflops_sustained": 1700.0}[kind], "of fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, path: str, index: int):
        self.path = path
        self.proc = None
        q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t_begin: float, t_end: float) -> dict:
        """Samples taken inside [t_begin, t_end] (wall clock); if the region
        was shorter than the sampling period, the samples nearest to it."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                ts = time.mktime(time.strptime(f[0].split(".")[0], "%Y/%m/%d %H:%M:%S")) + float("0." + f[0].split(".")[1])
                rows.append((ts, float(f[1]), float(f[2]), [n for n, v in zip(names, f[5:9])
                                                             if v.lower().startswith("active")]))
            except (ValueError, IndexError):
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        inside = [r for r in rows if t_begin <= r[0] <= t_end]
        where = "inside the timed region"
        if not inside:
            inside = sorted(rows, key=lambda r: min(abs(r[0] - t_begin), abs(r[0] - t_end)))[:3]
            where = "nearest to the timed region (shorter than the 200 ms sampling period)"
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": sorted({n for r in inside for n in r[3]}), "samples": len(inside), "where": where}


def oracle_slice_time(w, pairs, counter: str = "at", orc=None):
    """The CPU oracle on every host core (its multi-threaded calls: the pool
    split by row and frame range): ingest one whole slice, then the close
    (counts, loads, restore, NAT + Eq. 4) and the refresh.  Returns (seconds,
    cores, description, the oracle)."""
    import oracle
    if orc is None:
        orc = oracle.Oracle.from_params(w.params, mode={"at": 0, "ace": 1, "aligned": 2, "hist": 0}[counter])
    cores = oracle.cores()
    t0 = time.perf_counter()
    orc.ingest(pairs, threads=cores)
    orc.close_report(w.k, cap=1 << 16, threads=cores)
    orc.advance(threads=cores)
    dt = time.perf_counter() - t0
    text = ("oracle on %d host threads: ingest of one whole slice (%d pairs), its close (counts, loads, restore, "
            "NAT, Eq. 4) and refresh, %s workload, %s counters" % (cores, pairs.shape[0], w.name, counter.upper()))
    return dt, cores, text, orc


def line_config(w, args, world: int) -> dict:
    """The `config` of the main JSON line, the same for the device leg and
    the reference (oracle) leg of one command line."""
    return dict(workload_desc(w), counter=counter_for(args, w).upper(), key_table=args.key_table,
                cluster=args.cluster, parallelism="replicas" if world > 1 else "single",
                l2="inputs cycle over distinct slices held in memory, together larger than the L2 cache "
                   "(inputs_cycled); the pool state stays resident across steps")


def run_reference(args, w):
    """--impl reference: the oracle on every host core, each step one whole
    slice of the workload (the slices cycled as in the GPU leg)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_cycled = min(2, args.cycled or 2)
    host, _ = make_slices(w, n_cycled)
    times, pairs_done = [], 0
    text, cores, orc = "", 1, None
    for i in range(args.warmup + args.steps):
        p = host[i % n_cycled]
        dt, cores, text, orc = oracle_slice_time(w, p, counter_for(args, w), orc)
        if i >= args.warmup:
            times.append(dt)
            pairs_done += p.shape[0]
    total = sum(times)
    value = pairs_done / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pkts/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": line_config(w, args, int(os.environ.get("WORLD_SIZE", "1"))),
            "inputs_cycled": {"slices": n_cycled, "MB": sum(p.nbytes for p in host[:n_cycled]) >> 20},
            "cpu_baseline": {"value": value, "unit": "pkts/s", "cores": cores, "kind": "oracle", "sample": text},
            "e2e": {"value": value, "unit": "pkts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _slice_and_distinct(job):
    """Slice t of a workload and its number of distinct (aip, bip) pairs."""
    name, seed, t = job
    p = synth.workload(name, seed=seed).pairs(t)
    key = (p[:, 0].astype(np.uint64) << np.uint64(32)) | p[:, 1].astype(np.uint64)
    return p, int(np.unique(key).size)


def make_slices(w, n_slices: int):
    """The first n_slices slices of w, generated in parallel host processes
    (started with spawn, before any CUDA call of this process)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    jobs = [(w.name, w.seed, t) for t in range(n_slices)]
    if w.n_per_slice <= (1 << 20):
        res = [_slice_and_distinct(j) for j in jobs]
    else:
        with cf.ProcessPoolExecutor(max_workers=min(n_slices, os.cpu_count() or 1),
                                    mp_context=mp.get_context("spawn")) as ex:
            res = list(ex.map(_slice_and_distinct, jobs))
    return [r[0] for r in res], [r[1] for r in res]


def random_sector_rate(pool, stream, n_reads: int = 1 << 26, runs: int = 3) -> dict:
    """Random-access roofline: the rate of independent random 4-byte reads
    (one 32-byte sector each) of the pool's own words, CUDA events on the
    pool's stream, median of `runs` after one warm-up."""
    import torch
    pool.probe_random_reads(n_reads)
    ts = []
    for _ in range(runs):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        issued = pool.probe_random_reads(n_reads)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b) / 1e3)
    t = statistics.median(ts)
    l2 = getattr(torch.cuda.get_device_properties(torch.cuda.current_device()), "L2_cache_size", 0)
    return {"gbs": issued * 32 / t / 1e9, "reads_per_s": issued / t, "pool_bytes": 4 * pool.info()["pool_words"],
            "l2_bytes": int(l2)}


def reduce_over_ranks(times, counts, device):
    """Whole-job figures of the replicas: the slowest rank's times (max) and
    the units all ranks processed (sum)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x) for x in times], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(x) for x in counts], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return [float(x) for x in t] + [float(x) for x in c]


def stepwise_breakdown(pool, dev, w, n):
    """Mean device time of each stage of the stepwise close (scan, restore,
    refresh) next to the fused close, over n slices."""
    import torch
    stream = torch.cuda.current_stream()
    acc = {"ingest": [], "scan": [], "restore": [], "refresh": [], "fused_close": []}
    for i in range(n):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        e[0].record(stream)
        pool.ingest(dev[i % len(dev)])
        e[1].record(stream)
        pool.scan(w.k)
        e[2].record(stream)
        pool.restore()
        e[3].record(stream)
        pool.advance()
        e[4].record(stream)
        pool.report()
        for name, a, b in (("ingest", 0, 1), ("scan", 1, 2), ("restore", 2, 3), ("refresh", 3, 4)):
            acc[name].append(e[a].elapsed_time(e[b]))
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        pool.ingest(dev[(i + 1) % len(dev)])
        f0.record(stream)
        pool.close_slice(w.k)
        f1.record(stream)
        pool.report()
        acc["fused_close"].append(f0.elapsed_time(f1))
    return {k: statistics.mean(v) for k, v in acc.items()}


def gen_batch_gpu(n: int, seed: int, n_hosts: int = 1 << 20, alpha: float = 1.1):
    """n link-like (aip, bip) pairs generated on the GPU: Zipf(alpha) hosts,
    each with a bip set of size d drawn with P(D >= d) = 1/d (capped at 2^20).
    Returns an (n, 2) int32 CUDA tensor."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    ranks = torch.arange(1, n_hosts + 1, device="cuda", dtype=torch.float64)
    cdf = torch.cumsum(ranks ** (-alpha), 0)
    cdf /= cdf[-1].clone()
    rank = torch.searchsorted(cdf, torch.rand(n, generator=g, device="cuda", dtype=torch.float64))
    m32 = 0xFFFFFFFF

    def mix(x):
        x = x & m32
        x = x ^ (x >> 16)
        x = (x * 0x85EBCA6B) & m32
        x = x ^ (x >> 13)
        x = (x * 0xC2B2AE35) & m32
        return x ^ (x >> 16)
    aip = mix(rank + seed * 7919)
    u = (mix(rank ^ 0x2545F491) + 1).double() / 4294967297.0
    d = torch.clamp(torch.floor(1.0 / u), max=float(1 << 20))
    j = torch.floor(torch.rand(n, generator=g, device="cuda", dtype=torch.float64) * d).long()
    bip = mix(mix(aip ^ 0x5BD1E995) + j)
    out = torch.stack([aip, bip], dim=1)
    return torch.where(out >= (1 << 31), out - (1 << 32), out).to(torch.int32).contiguous()


def learned_accuracy(asse, w, stream, torch, loss_kind: str = "rel_mse", n_train: int = 1_800_000,
                     n_test: int = 200_000, n_max_log2: int = 20, bg_max: float = 0.08, epochs: int = 3):
    """Train the model on synthetic states shaped like w's ATVs (the GPU
    generator and training kernels): n_train states with cardinality
    log-uniform in [1, 2^n_max_log2] spread over the window, background up to
    bg_max per AT and slice; then the mean relative error on n_test held-out
    states, over the whole range and by range of the true cardinality, for
    the model alone, for the learned estimate with its Eq. 2 fallback, and
    for Eq. 2 alone."""
    keys = synth.method_keys(1)
    scfg = dict(k=w.k, g=w.g, r=w.r, n_max_log2=n_max_log2, bg_max=bg_max, seed=11, bh_a=keys["bh_a"],
                bh_b=keys["bh_b"])
    xs, lns, _lcs = asse.synth_states(scfg, 0, n_train, stream=stream.cuda_stream)
    xt, lnt, lct = asse.synth_states(scfg, 1 << 40, n_test, stream=stream.cuda_stream)
    trained = asse.MLP(seed=2, stream=stream.cuda_stream)
    trained.set_loss(loss_kind)
    gen = torch.Generator(device="cuda").manual_seed(0)
    bs = 4096
    n_steps = epochs * (n_train // bs)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    perm = None
    for step in range(n_steps):
        o = (step * bs) % (n_train - n_train % bs)
        if o == 0:
            perm = torch.randperm(n_train, device="cuda", generator=gen)
        idx = perm[o:o + bs]
        lr = 2e-3 if step < 0.6 * n_steps else (5e-4 if step < 0.85 * n_steps else 1e-4)
        trained.train_step(xs[idx].contiguous(), lns[idx].contiguous(), lr)
    t1.record(stream)
    yt = trained.forward(xt)
    trained.check()
    n_true = torch.exp(lnt.double())
    lnmax = n_max_log2 * float(np.log(2.0))
    cnt = xt[:, 0].double() * w.g
    # the rule of asse_estimate_learned: the model unless the ATV is empty or
    # the model is above its training range; then Eq. 2
    inside = (cnt > 0.5) & (yt <= lnmax)
    est_mlp = torch.exp(yt.double())
    est_rule = torch.where(inside, torch.exp(torch.clamp(yt.double(), min=0.0)), lct.double())
    rel = {name: (torch.abs(e - n_true) / n_true) for name, e in
           (("mlp", est_mlp), ("learned_with_fallback", est_rule), ("eq2", lct.double()))}
    bins = {}
    edges = [0, 4, 8, 12, 16, n_max_log2 + 1]
    lg = lnt.double() / np.log(2.0)
    for a, b in zip(edges[:-1], edges[1:]):
        sel = (lg >= a) & (lg < b)
        if int(sel.sum()) == 0:
            continue
        bins["2^%d..2^%d" % (a, min(b, n_max_log2))] = {k: v[sel].mean().item() for k, v in rel.items()}
    return {"states": "k=%d, g=%d, r=%d, cardinalities log-uniform in [1, 2^%d] spread over the window with random "
                      "shares, background up to %.2f per AT and slice; %d training and %d held-out states"
                      % (w.k, w.g, w.r, n_max_log2, bg_max, n_train, n_test),
            "loss": loss_kind, "train_rows": n_steps * bs, "train_ms": t0.elapsed_time(t1),
            "mre": {k: v.mean().item() for k, v in rel.items()}, "mre_by_range": bins,
            "fallback_fraction": 1.0 - inside.double().mean().item()}


def run_learned(args):
    """Per-slice learned inference: the feature rows of every ATV of a
    scanned pool (r x E rows) and the MLP on them (tcgen05 kernel).  The
    features and the model are re-run on the same scanned state each step."""
    import torch
    from paper_1807_01527_gb300 import asse, build
    build.build()
    w = synth.workload(args.workload, seed=1)
    stream = torch.cuda.current_stream()
    counter = counter_for(args, w)
    pool = asse.Pool(w.params, counter=counter, stream=stream.cuda_stream)
    pairs = w.pairs(0) if w.n_per_slice <= (8 << 20) else gen_batch_gpu(w.n_per_slice, 3, w.n_hosts, w.zipf)
    src = torch.from_numpy(pairs.view(np.int32)).cuda() if isinstance(pairs, np.ndarray) else pairs
    pool.ingest(src)
    pool.scan(w.k)
    model = asse.MLP(seed=1, stream=stream.cuda_stream)
    rows = w.r << w.E_log2
    x = pool.features()
    y = torch.empty(rows, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        pool.features()
        model.forward(x, y)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = Clocks(os.path.join(tempfile.gettempdir(), "bench_clocks_learned.csv"), 0)
    wall0 = time.time()
    for i in range(args.steps):
        ev[i][0].record(stream)
        xi = pool.features()
        ev[i][1].record(stream)
        model.forward(xi, y)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    wall1 = time.time()
    model.check()
    t_feat = statistics.mean(ev[i][0].elapsed_time(ev[i][1]) for i in range(args.steps)) / 1e3
    t_mlp = statistics.mean(ev[i][1].elapsed_time(ev[i][2]) for i in range(args.steps)) / 1e3
    peak, src_peak = peaks("bf16_tflops")
    achieved = rows * MLP_FLOP_PER_ROW / t_mlp / 1e12
    # accuracy on the learned-estimator workload: link-shaped states (k=10, g=512)
    wl = synth.workload("link", seed=1)
    acc = None if args.no_accuracy else {kind: learned_accuracy(asse, wl, stream, torch, kind)
                                         for kind in ("rel_mse", "log_mse")}
    line = {"metric": "learned per-ATV inference: feature rows + MLP per scanned slice", "value": rows / (t_feat + t_mlp),
            "unit": "rows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "mode": "learned",
            "ms_per_step": 1e3 * (t_feat + t_mlp), "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
            "config": dict(workload_desc(w), rows_per_step=rows, counter=counter.upper(),
                           features=("from the slice counts (k' per ATV)" if counter == "hist" else
                                     "from the pool words"),
                           l2="feature rows %d MB (%s the 129 MB L2), re-read each step"
                              % (rows * 160 >> 20, "within" if rows * 160 < (100 << 20) else "larger than")),
            "kernel_ms": {"features": 1e3 * t_feat, "mlp_tcgen05": 1e3 * t_mlp},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "mlp_forward (tcgen05)",
                         "peak_source": src_peak + " (bf16 burst)",
                         "model": "2 x (68 x 256 + 256 x 256 + 256) FLOP per row"},
            "accuracy": acc,
            "clocks": clocks.stop(wall0, wall1)}
    print(json.dumps(line), flush=True)
    pool.close()


def run_serve(args):
    """Serving: 16 independent streams (k in {4,10,30,60}, 2^14..2^18 ATVs per
    row, g in {128,512,1024}), slice batches of exponential size with mean 4 Mi
    pairs clipped to [64 Ki, 16 Mi], a 20 GB device-memory budget; every stream
    always has its next batch ready (closed loop), each batch followed by the
    close of its slice.  Reports aggregate pairs/s and the p50/p99 device
    latency from the start of a close to its report in host memory."""
    import torch
    from paper_1807_01527_gb300 import asse, build
    build.build()
    rng = np.random.default_rng(5)
    n_streams, slices_per_stream = 16, args.serve_slices
    streams = []
    for i in range(n_streams):
        k = int(rng.choice([4, 10, 30, 60]))
        g = int(rng.choice([128, 512, 1024]))
        g = max(g, 2 * k)
        elog = int(rng.integers(14, 19))
        c, u, s_ = synth.column_split(elog, 4)
        p = dict(k=k, theta=g, g=g, r=4, c=c, u=u, s=s_, **synth.method_keys(1000 + i))
        sizes = np.clip(rng.exponential(4 << 20, size=slices_per_stream), 64 << 10, 16 << 20).astype(np.int64)
        streams.append((p, sizes))
    # batches: a few distinct GPU-generated batches per stream, reused across its slices
    pool_of_batches = {}
    for i, (p, sizes) in enumerate(streams):
        uniq = sorted(set(int(x) for x in sizes[:3]))
        for n in uniq:
            pool_of_batches[(i, n)] = gen_batch_gpu(n, 31 * i + n % 997)
    torch.cuda.synchronize()

    def batch_for(i, t):
        sizes = streams[i][1]
        n = int(sizes[t])
        key = (i, n) if (i, n) in pool_of_batches else min((kk for kk in pool_of_batches if kk[0] == i),
                                                          key=lambda kk: abs(kk[1] - n))
        return pool_of_batches[key]

    srv = asse.Server(20 << 30)
    model = None
    if args.serve_learned:
        # learned per-ATV inference inside every close graph (one model for all streams)
        model = asse.MLP(seed=1, stream=torch.cuda.current_stream().cuda_stream)
        model.set_loss("rel_mse")
    waiting = list(range(n_streams))
    running = {}
    lat, pairs_done, deferred, max_open = [], 0, 0, 0
    host_s = {"open": 0.0, "submit": 0.0, "poll": 0.0, "close": 0.0}
    overflowed = 0
    # the interval in which every admitted stream is open and none has closed yet
    t_all_open, t_first_close, pairs_steady = None, None, 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while waiting or running:
        while waiting:
            i = waiting[0]
            sp = streams[i][0]
            ctr = args.counter if args.counter != "auto" else auto_counter(sp["k"], sp["g"], sp["r"], sp["c"] + sp["u"])
            th = time.perf_counter()
            sid = srv.open(sp, sp["k"], max_batch=16 << 20, counter=ctr)
            host_s["open"] += time.perf_counter() - th
            if sid is None:
                deferred += 1
                break
            waiting.pop(0)
            if model is not None:
                srv.attach_model(sid, model, 20 * float(np.log(2.0)))
            running[i] = [sid, 0, 0]          # sid, slices submitted, slices reported
        max_open = max(max_open, len(running))
        if not waiting and t_all_open is None:
            t_all_open = time.perf_counter()
        progressed = False
        for i in list(running):
            sid, sub, rep = running[i]
            # submit only into a free report slot, poll only a stream with a
            # close in flight: a call that can only answer "again" still
            # costs the loop its host time
            if sub < slices_per_stream and sub - rep < asse.SERVE_RING:
                b = batch_for(i, sub)
                th = time.perf_counter()
                ok = srv.submit(sid, b, close=True)
                host_s["submit"] += time.perf_counter() - th
                if ok:
                    running[i][1] += 1
                    pairs_done += b.shape[0]
                    progressed = True
            if running[i][1] == running[i][2]:
                continue
            th = time.perf_counter()
            try:
                r = srv.poll(sid)
            except asse.AsseError as ex:
                # a saturated small pool: more candidates than the restore
                # capacity; the close is done and its report incomplete
                if ex.status != asse.ECAPACITY:
                    raise
                r = "overflow"
            host_s["poll"] += time.perf_counter() - th
            if r is not None:
                if r == "overflow":
                    overflowed += 1
                else:
                    lat.append(r[2])
                if t_all_open is not None and t_first_close is None:
                    pairs_steady += batch_for(i, running[i][2]).shape[0]
                running[i][2] += 1
                progressed = True
            if running[i][2] == slices_per_stream:
                if t_first_close is None:
                    t_first_close = time.perf_counter()
                th = time.perf_counter()
                srv.close(sid)
                host_s["close"] += time.perf_counter() - th
                del running[i]
        if not progressed:
            time.sleep(20e-6)
    srv.sync()
    wall = time.perf_counter() - t0
    srv.destroy()
    lat.sort()
    line = {"metric": "serving: aggregate pkts/s over 16 streams, p50/p99 slice-close-to-report latency",
            "value": pairs_done / wall, "unit": "pkts/s", "n_gpus": 1, "higher_is_better": True,
            "mode": "serve", "dtype": "u32", "data": "synthetic",
            "config": {"workload": "16 streams, k in {4,10,30,60}, 2^14..2^18 ATVs/row, g in {128,512,1024}, "
                                   "batches exp(mean 4Mi) clipped [64Ki,16Mi], 20 GB budget",
                       "counter": args.counter.upper() + (" (slice counts for pools larger than L2)"
                                                          if args.counter == "auto" else ""),
                       "slices_per_stream": slices_per_stream},
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "what": "device time from the start of a close to its report in host memory"},
            "pairs": pairs_done, "wall_s": wall, "closes": len(lat), "admission_deferrals": deferred,
            "max_streams_open": max_open,
            "host_ms_in_calls": {k: 1e3 * v for k, v in host_s.items()},
            "closes_over_restore_capacity": overflowed,
            "steady": {"value": pairs_steady / (t_first_close - t_all_open)
                       if t_all_open is not None and t_first_close is not None and t_first_close > t_all_open
                       else None, "unit": "pkts/s",
                       "what": "pairs of the closes reported while every admitted stream was open and none had "
                               "closed yet, over that interval (no stream opening or closing in it)"},
            "learned_inference_in_close": bool(args.serve_learned)}
    print(json.dumps(line), flush=True)


def _slice_and_keys(job):
    """Slice t of a workload and its distinct (aip, bip) keys (a spawned
    worker of the accuracy leg)."""
    from oracle import truth
    name, seed, t = job
    p = synth.workload(name, seed=seed).pairs(t)
    return p, truth.slice_keys(p)


def _rates_summary(rows: list) -> dict:
    """Mean FPR / FNR / FTR over the windows that hold super points."""
    rows = [r for r in rows if r["fpr"] is not None]
    if not rows:
        return {"windows": 0}
    return {"windows": len(rows), "fpr": statistics.mean(r["fpr"] for r in rows),
            "fnr": statistics.mean(r["fnr"] for r in rows), "ftr": statistics.mean(r["ftr"] for r in rows),
            "super_points_mean": statistics.mean(r["n"] for r in rows)}


def run_accuracy(args):
    """Detection accuracy on the workload's ground truth (exact window
    cardinalities, Sec. 2.1), as FPR / FNR / FTR (Sec. 5), of:
      - the sliding pool with Eq. 4 (the paper's method), every slice;
      - the same candidates decided by the learned candidate model instead of
        Eq. 4 (trained here on synthetic candidate states shaped like the
        pool: k, g, r and the row loads the first window shows);
      - the discrete-window mode (1-bit aging counters, k = 1, reset after
        every window of k slices) at equal memory: the same words per ATV,
        so 32 x words ATs of one bit each, read at the end of each window."""
    import concurrent.futures as cf
    import multiprocessing as mp
    w = synth.workload(args.workload, seed=1)
    k = w.k
    T = args.acc_slices or (3 * k if w.n_per_slice <= (8 << 20) else k + 3)
    ex = cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn"))
    futs = [ex.submit(_slice_and_keys, (w.name, w.seed, t)) for t in range(T)]

    import torch
    from oracle import truth
    from paper_1807_01527_gb300 import asse, build
    build.build()
    stream = torch.cuda.current_stream()
    sliding = asse.Pool(w.params, stream=stream.cuda_stream, restore_cap=1 << 14)
    words = sliding.info()["words"]
    p1 = dict(w.params, k=1, g=32 * words)
    discrete = asse.Pool(p1, counter="ace", stream=stream.cuda_stream, restore_cap=1 << 14)
    mem = {"sliding_bytes": 4 * sliding.info()["pool_words"], "discrete_bytes": 4 * discrete.info()["pool_words"],
           "sliding": "g=%d ATs of %d bits" % (w.g, sliding.info()["w"]),
           "discrete": "g=%d ATs of 1 bit (k=1 aging counters, reset every %d slices)" % (p1["g"], k)}
    keys, model, model_info = [], None, None
    max_log_n = 20 * float(np.log(2.0))
    res = {"eq4": [], "learned": [], "discrete": []}
    t0 = time.time()
    for t in range(T):
        pairs, kt = futs[t].result()
        keys.append(kt)
        dev = torch.from_numpy(pairs.view(np.int32)).cuda()
        sliding.ingest(dev)
        discrete.ingest(dev)
        del pairs
        sliding.scan(k)
        if model is None and t == k - 1:
            # row loads of the first full window -> background of the training states
            P = sliding.loads().astype(np.float64) / (w.g * (1 << w.c))
            p_slice = 1.0 - (1.0 - float(P.max())) ** (1.0 / k)
            model, model_info = train_candidate_model(asse, w, stream, torch, bg_max=min(1.0, 2.0 * p_slice),
                                                      n_max_log2=20)
        sliding.restore()
        cand = sliding.candidates()
        if t >= k - 1:
            true_sp = truth.super_points(keys[t - k + 1:t + 1], w.theta)
            res["eq4"].append(truth.error_rates({int(a) for a in cand["aip"][cand["est"] >= w.theta]}, true_sp))
            # the same candidates decided on the device by the learned model
            # (Eq. 4 where the model's output leaves its training range)
            learned = {int(a) for a in sliding.report_learned(model, max_log_n)["aip"]}
            res["learned"].append(truth.error_rates(learned, true_sp))
        sliding.advance()
        if (t + 1) % k == 0:
            discrete.close_slice(1)
            rep = discrete.report()
            res["discrete"].append(truth.error_rates({int(a) for a in rep["aip"]},
                                                     truth.super_points(keys[t - k + 1:t + 1], w.theta)))
        if t >= k:
            keys[t - k] = None
    ex.shutdown()
    line = {"metric": "detection accuracy on exact window cardinalities: FPR, FNR, FTR (Sec. 5)", "mode": "accuracy",
            "config": dict(workload_desc(w), slices=T), "data": "synthetic",
            "sliding_eq4": _rates_summary(res["eq4"]), "sliding_learned_candidates": _rates_summary(res["learned"]),
            "discrete_1bit_equal_memory": _rates_summary(res["discrete"]), "memory": mem,
            "candidate_model": model_info, "wall_s": time.time() - t0,
            "per_window": {kk: [(r["n"], r["n_plus"], r["n_minus"]) for r in v] for kk, v in res.items()}}
    print(json.dumps(line), flush=True)


def train_candidate_model(asse, w, stream, torch, bg_max: float, n_max_log2: int = 20, n_train: int = 1_200_000,
                          n_test: int = 100_000, epochs: int = 3):
    """The learned replacement of Eq. 4: an MLP trained with the relative
    loss on synthetic candidate states of w's shape (k, g, r), background up
    to bg_max per AT and slice in each row.  Returns (model, summary with the
    held-out mean relative error of the model and of Eq. 4)."""
    keys = synth.method_keys(w.seed)
    cfg = dict(k=w.k, g=w.g, r=w.r, n_max_log2=n_max_log2, bg_max=bg_max, seed=41, bh_a=keys["bh_a"],
               bh_b=keys["bh_b"])
    x, ln, _e4 = asse.synth_candidates(cfg, 0, n_train, stream=stream.cuda_stream)
    xt, lnt, e4t = asse.synth_candidates(cfg, 1 << 40, n_test, stream=stream.cuda_stream)
    m = asse.MLP(seed=6, stream=stream.cuda_stream)
    m.set_loss("rel_mse")
    gen = torch.Generator(device="cuda").manual_seed(2)
    bs = 4096
    n_steps = epochs * (n_train // bs)
    perm = None
    for step in range(n_steps):
        o = (step * bs) % (n_train - n_train % bs)
        if o == 0:
            perm = torch.randperm(n_train, device="cuda", generator=gen)
        idx = perm[o:o + bs]
        lr = 2e-3 if step < 0.6 * n_steps else (5e-4 if step < 0.85 * n_steps else 1e-4)
        m.train_step(x[idx].contiguous(), ln[idx].contiguous(), lr)
    y = m.forward(xt)
    m.check()
    n_true = torch.exp(lnt.double())
    e4 = torch.where(torch.isinf(e4t), torch.full_like(e4t, 1e12), e4t).double()
    rel_m = torch.abs(torch.exp(y.double()) - n_true) / n_true
    rel_e = torch.abs(e4 - n_true) / n_true
    near = (lnt >= np.log(w.theta / 4.0)) & (lnt < np.log(4.0 * w.theta))
    # Eq. 4 is infinite once NAT = g: the mean relative error is then
    # meaningless, so the median and the share within 10 % are given too
    return m, {"states": "k=%d, g=%d, r=%d, cardinalities log-uniform in [1, 2^%d], per-row background up to %.4f "
                         "per AT and slice; %d training, %d held-out" % (w.k, w.g, w.r, n_max_log2, bg_max, n_train,
                                                                         n_test),
               "mre_model": rel_m.mean().item(), "mre_eq4": rel_e.mean().item(),
               "median_rel_model": rel_m.median().item(), "median_rel_eq4": rel_e.median().item(),
               "within_10pct_model": (rel_m <= 0.1).double().mean().item(),
               "within_10pct_eq4": (rel_e <= 0.1).double().mean().item(),
               "near_theta": {"range": "theta/4 .. 4 theta",
                              "median_rel_model": rel_m[near].median().item(),
                              "median_rel_eq4": rel_e[near].median().item(),
                              "within_10pct_model": (rel_m[near] <= 0.1).double().mean().item(),
                              "within_10pct_eq4": (rel_e[near] <= 0.1).double().mean().item()}}


def scan_alg_bytes(w, pool_info: dict, counter: str, kp: int | None = None) -> float:
    """Algorithmic bytes of one fused scan: the pool read once, plus the words
    the refresh rewrites: the two ACT blocks whose ACT becomes 0 or k (2 of
    the 2k blocks of every ATV, Algorithm 2) for timestamps, every word
    every k slices for the aligned variant (averaged per slice), every word
    for aging counters."""
    pool_bytes = 4.0 * pool_info["pool_words"]
    if counter == "hist":
        # per ATV: its window sum read and written back, the count of the
        # phase leaving the window read, the opening phase's count zeroed (2
        # bytes each; a window shorter than k reads its k' counts instead of
        # the sum); the refresh of the two checked blocks, fused into the same
        # kernel, reads their words
        kp = w.k if kp is None else kp
        per_atv = 8.0 if kp == w.k else 2.0 * kp + 8.0
        return per_atv * w.r * pool_info["E"] + pool_bytes * 2.0 / (2 * w.k)
    if counter == "ace":
        return 2 * pool_bytes
    if counter == "aligned":
        return pool_bytes * (1.0 + 1.0 / w.k)
    return pool_bytes * (1.0 + 2.0 / (2 * w.k))


def roofline_entry(kernel: str, alg_bytes: float, t_s: float, peak: float, peak_src: str, model: str,
                   workload: str, counter: str) -> dict:
    traffic, capture, current = traffic_of(workload, counter, kernel)
    achieved = alg_bytes / t_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_capture": capture if current else None,
            "kernel": kernel, "peak_source": peak_src, "algorithmic_bytes_per_launch": alg_bytes,
            "ms_per_launch": 1e3 * t_s, "model": model}


def auto_counter(k: int, g: int, r: int, E_log2: int) -> str:
    """Timestamps with slice counts for a pool larger than the L2 cache (the
    close then reads 2 bytes per ATV and slice instead of the pool), plain
    timestamps for one that fits (its ingest would pay the slice counts'
    atomics for a close that is already fast)."""
    w = max(1, (2 * k).bit_length())          # ceil(log2(2k + 1))
    w = 8 if w == 7 else w
    words = -(-(-(-g // (32 // w))) // 8) * 8
    return "hist" if 4 * r * (1 << E_log2) * words > (128 << 20) else "at"


def counter_for(args, w) -> str:
    """The counter kind of a workload: --counter, or auto_counter's choice."""
    if args.counter != "auto":
        return args.counter
    return auto_counter(w.k, w.g, w.r, w.E_log2)


def bench_workload(w, args, world, rank, stream, torch, asse, dist, with_e2e=True):
    """One workload: ingest + fused close per step, device-timed over
    args.steps steps with inputs resident in HBM, then end to end from pinned
    host buffers.  Returns the measurements (rank-local times and counts)."""
    n_cycled = args.cycled or (N_SLICES_CYCLED if w.n_per_slice <= (8 << 20) else 4)
    host, n_distinct = args.slices_of(w, n_cycled)
    dev = [torch.from_numpy(p.view(np.int32)).cuda() for p in host]
    pinned = [torch.from_numpy(p.view(np.int32)).pin_memory() for p in host] if with_e2e else None
    n_pairs = [p.shape[0] for p in host]
    counter = counter_for(args, w)
    pool = asse.Pool(w.params, counter=counter, stream=stream.cuda_stream, key_table=args.key_table,
                     cluster=args.cluster)

    for i in range(args.warmup):
        pool.ingest(dev[i % n_cycled])
        pool.close_slice(w.k)
        pool.report()
    torch.cuda.synchronize()

    # device-timed region: inputs resident, per-kernel events on the pool stream
    pool.set_timing(True)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    lat, t_scan, t_restore = [], [], []
    launches0 = pool.launches
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.time()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    pairs_done, n_reported = 0, 0
    # Step i: ingest slice i, close it, read its report on the host.  The
    # next slice's ingest is queued before the report is read (the report
    # waits for its own close only), so the device does not idle while the
    # host reads.
    host_t = {"ingest_call": [], "close_call": [], "report_call": []}

    def src_of(i):
        return dev[(args.warmup + i) % n_cycled]
    ev[0][0].record(stream)
    pool.ingest(src_of(0))
    ev[0][1].record(stream)
    for i in range(args.steps):
        t0 = time.perf_counter()
        pool.close_slice(w.k)
        ev[i][2].record(stream)
        t1 = time.perf_counter()
        if i + 1 < args.steps:
            ev[i + 1][0].record(stream)
            pool.ingest(src_of(i + 1))
            ev[i + 1][1].record(stream)
        h1 = time.perf_counter()
        rep = pool.report()
        t2 = time.perf_counter()
        sc, rs = pool.close_timing()
        t_scan.append(sc / 1e3)
        t_restore.append(rs / 1e3)
        lat.append(t2 - t0)
        host_t["close_call"].append(t1 - t0)
        host_t["ingest_call"].append(h1 - t1)
        host_t["report_call"].append(t2 - h1)
        n_reported += rep.size
        pairs_done += n_pairs[(args.warmup + i) % n_cycled]
    end.record(stream)
    torch.cuda.synchronize()
    elapsed = start.elapsed_time(end) / 1e3
    launches = pool.launches - launches0
    if world > 1:
        dist.barrier()
    wall1 = time.time()
    pool.set_timing(False)
    t_ingest = [ev[i][0].elapsed_time(ev[i][1]) / 1e3 for i in range(args.steps)]
    t_close = [ev[i][1].elapsed_time(ev[i][2]) / 1e3 for i in range(args.steps)]

    # end to end through the public API with host buffers: pinned pairs ->
    # device (asse_ingest returns once the buffer has been read) -> ingest ->
    # close -> report on the host; as in the device-timed loop, the next
    # slice's pairs go in before the report of this one is read
    e2e_pairs, d2h, e2e_elapsed = 0, 0, None
    if with_e2e:
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        pool.ingest(pinned[args.warmup % n_cycled])
        for i in range(args.steps):
            j = (args.warmup + i) % n_cycled
            pool.close_slice(w.k)
            if i + 1 < args.steps:
                pool.ingest(pinned[(args.warmup + i + 1) % n_cycled])
            rep = pool.report()
            e2e_pairs += n_pairs[j]
            d2h += rep.nbytes + 32
        torch.cuda.synchronize()
        e2e_elapsed = time.perf_counter() - t0
    breakdown = stepwise_breakdown(pool, dev, w, args.warmup) if args.breakdown else None
    sector = random_sector_rate(pool, stream)
    used = [(args.warmup + i) % n_cycled for i in range(args.steps)]
    info = pool.info()
    pool.close()
    return dict(elapsed=elapsed, e2e_elapsed=e2e_elapsed, pairs_done=pairs_done, e2e_pairs=e2e_pairs, d2h=d2h,
                t_ingest=t_ingest, t_close=t_close, t_scan=t_scan, t_restore=t_restore, lat=lat, host_t=host_t,
                launches=launches, n_reported=n_reported, wall=(wall0, wall1), breakdown=breakdown, sector=sector,
                used=used, n_pairs=n_pairs, n_distinct=n_distinct, host=host, info=info, n_cycled=n_cycled)


def summarize(w, args, m) -> dict:
    """Kernel times, latencies and the rooflines of the ingest and the scan."""
    ing = statistics.mean(m["t_ingest"])
    scan = statistics.mean(m["t_scan"])
    used = m["used"]
    peak, peak_src = peaks()
    alg_ing = statistics.mean(8 * m["n_pairs"][j] + 32 * w.r * m["n_distinct"][j] for j in used)
    counter = counter_for(args, w)
    alg_scan = scan_alg_bytes(w, m["info"], counter)
    r_ing = roofline_entry("ingest", alg_ing, ing, peak, peak_src,
                           "8 B per pair + 32 B x r per distinct (aip, bip) pair", w.name, counter)
    r_ing["distinct_pair_fraction"] = statistics.mean(m["n_distinct"][j] / m["n_pairs"][j] for j in used)
    r_scan = roofline_entry("hist_scan" if counter == "hist" else "scan", alg_scan, scan, peak, peak_src,
                            "per ATV its window sum read and written, the leaving and the opening phase's "
                            "counts (2 B each) + the words of the two refreshed blocks" if counter == "hist" else
                            "the pool read once + the refreshed words written (Algorithm 2)", w.name, counter)
    lat_ms = sorted(1e3 * x for x in m["lat"])
    sector = m["sector"]
    return {
        "kernel_ms": {"ingest": 1e3 * ing, "close": 1e3 * statistics.mean(m["t_close"]), "scan": 1e3 * scan,
                      "restore": 1e3 * statistics.mean(m["t_restore"]),
                      "ingest_p50": 1e3 * statistics.median(m["t_ingest"]),
                      "close_p50": 1e3 * statistics.median(m["t_close"]),
                      "what": "CUDA events on the pool's stream: around each ingest and close call, and recorded by "
                              "the library around the scan and the restore kernel of each close"},
        "slice_latency_ms": {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[min(len(lat_ms) - 1,
                                                                                 int(0.99 * len(lat_ms)))],
                             "what": "close_slice call to report on the host (the next slice's ingest is "
                                     "queued in between)"},
        "rooflines": {"ingest": r_ing, "scan": r_scan},
        "random_sector_roofline": {
            "peak": sector["gbs"], "unit": "GB/s", "frac": r_ing["achieved"] / sector["gbs"],
            "reads_per_s": sector["reads_per_s"],
            "what": "random 4-byte reads of this pool's words (one 32-byte sector each, every SM busy), "
                    "timed in this run (pool of %d MB, L2 of %d MB); the ingest's algorithmic bytes per launch "
                    "over its time, against this rate" % (sector["pool_bytes"] >> 20, sector["l2_bytes"] >> 20)},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="long", choices=["tiny_b", "link", "long"],
                    help="the headline workload (default: the long window, k=60, 32 Mi pairs per slice)")
    ap.add_argument("--secondary", default="link", choices=["link", "none"],
                    help="a second workload measured in the same run and reported under its own key")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--breakdown", action="store_true", help="also time scan / restore / refresh separately")
    ap.add_argument("--mode", default="slice", choices=["slice", "serve", "learned", "accuracy"],
                    help="slice: one pool, the headline line; serve: the multi-stream serving loop; "
                         "learned: per-slice learned inference (features + tensor-core MLP); accuracy: FPR/FNR of "
                         "the sliding pool (Eq. 4 and the learned candidate model) and of the 1-bit discrete mode "
                         "at equal memory, on exact window cardinalities")
    ap.add_argument("--acc-slices", type=int, default=0, help="accuracy mode: slices to run (0: 3k, or k+3 for the "
                                                              "long workload)")
    ap.add_argument("--serve-slices", type=int, default=12)
    ap.add_argument("--serve-learned", action="store_true",
                    help="serve mode: run learned per-ATV inference inside every close graph")
    ap.add_argument("--no-accuracy", action="store_true", help="learned mode: skip the training and accuracy leg")
    ap.add_argument("--cycled", type=int, default=0,
                    help="distinct input slices cycled through (0: 8, or 4 for slices over 8 Mi pairs)")
    ap.add_argument("--key-table", default="auto", choices=["auto", "on", "off"],
                    help="the ingest's slice-wide key table (auto: for pools larger than L2)")
    ap.add_argument("--clocks-dir", default="", help="where the nvidia-smi clock samples of the timed region go "
                                                      "(default: the temporary directory)")
    ap.add_argument("--counter", default="auto", choices=["auto", "at", "ace", "aligned", "hist"],
                    help="at: the paper's asynchronous timestamps; ace: aging counters; aligned: timestamps with "
                         "one ACT per ATV (whole-pool refresh every k slices); hist: timestamps with per-ATV slice "
                         "counts kept by the ingest (the close reads the counts); auto: hist for a pool larger "
                         "than L2, else at")
    ap.add_argument("--cluster", type=int, default=0, choices=[0, 1, 2, 4, 8],
                    help="CTAs of a thread-block cluster sharing the ingest's table of seen keys (0: the library's "
                         "choice)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.mode in ("serve", "learned", "accuracy"):
        if rank == 0:
            {"serve": run_serve, "learned": run_learned, "accuracy": run_accuracy}[args.mode](args)
        return
    w = synth.workload(args.workload, seed=1 + rank)
    if args.impl == "reference":
        run_reference(args, w)
        return
    w2 = None
    if args.secondary != "none" and args.secondary != args.workload:
        w2 = synth.workload(args.secondary, seed=1 + rank)

    # every input slice is generated up front, in host processes started with
    # spawn before any CUDA call of this process
    pre = {}
    for wl in (w, w2):
        if wl is not None:
            nc = args.cycled or (N_SLICES_CYCLED if wl.n_per_slice <= (8 << 20) else 4)
            pre[wl.name] = make_slices(wl, nc)
    args.slices_of = lambda wl, n: pre[wl.name]

    import torch
    from paper_1807_01527_gb300 import asse, build
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    stream = torch.cuda.current_stream()

    clocks = Clocks(os.path.join(args.clocks_dir or tempfile.gettempdir(), "bench_clocks_%d.csv" % rank), local)
    m = bench_workload(w, args, world, rank, stream, torch, asse, dist)
    clk = clocks.stop(*m["wall"])
    m2 = bench_workload(w2, args, world, rank, stream, torch, asse, dist) if w2 is not None else None

    elapsed, e2e_elapsed, pairs_done, e2e_pairs = m["elapsed"], m["e2e_elapsed"], m["pairs_done"], m["e2e_pairs"]
    if world > 1:
        elapsed, e2e_elapsed, pairs_done, e2e_pairs = reduce_over_ranks([elapsed, e2e_elapsed],
                                                                        [pairs_done, e2e_pairs], "cuda")
    second = None
    if m2 is not None:
        el2, pd2 = m2["elapsed"], m2["pairs_done"]
        ee2, ep2 = m2["e2e_elapsed"], m2["e2e_pairs"]
        if world > 1:
            el2, ee2, pd2, ep2 = reduce_over_ranks([el2, ee2], [pd2, ep2], "cuda")
        second = dict(summarize(w2, args, m2), value=pd2 / el2, unit="pkts/s",
                      ms_per_step=1e3 * el2 / args.steps,
                      config=dict(workload_desc(w2), counter=counter_for(args, w2).upper()),
                      e2e={"value": ep2 / ee2, "unit": "pkts/s",
                           "h2d_bytes_per_step": int(8 * statistics.mean(m2["n_pairs"])),
                           "d2h_bytes_per_step": int(m2["d2h"] / args.steps)})

    if rank == 0:
        summ = summarize(w, args, m)
        rl = summ.pop("rooflines")
        dominant = max(rl, key=lambda k: rl[k]["ms_per_launch"])
        line = {
            "metric": METRIC, "value": pairs_done / elapsed, "unit": "pkts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": line_config(w, args, world),
            "inputs_cycled": {"slices": m["n_cycled"], "MB": sum(p.nbytes for p in m["host"]) >> 20},
            "roofline": dict(rl[dominant], dominant=True),
            "roofline_other": {k: v for k, v in rl.items() if k != dominant},
            "e2e": {"value": e2e_pairs / e2e_elapsed, "unit": "pkts/s",
                    "h2d_bytes_per_step": int(8 * statistics.mean(m["n_pairs"])),
                    "d2h_bytes_per_step": int(m["d2h"] / args.steps)},
            "gpu_launches": int(m["launches"]),
            "reported_per_slice": m["n_reported"] / args.steps,
            "host_call_ms_p50": {k: 1e3 * statistics.median(v) for k, v in m["host_t"].items()},
            "clocks": clk,
        }
        line.update(summ)
        if m["breakdown"]:
            line["breakdown_ms"] = m["breakdown"]
        if second is not None:
            line[w2.name] = second
        if not args.no_cpu_baseline and world == 1:
            p0 = m["host"][0]
            dt, cores, text, _ = oracle_slice_time(w, p0, counter_for(args, w))
            line["cpu_baseline"] = {"value": p0.shape[0] / dt, "unit": "pkts/s", "cores": cores, "kind": "oracle",
                                    "sample": text}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
