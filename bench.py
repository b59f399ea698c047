#!/usr/bin/env python3
"""Benchmark of the eager sparse BM25 hot path on one GB300.

One step = the whole hot path over one batch of synthetic input:
index build from device-resident tokens (|D|, TF, DF, IDF, S0, CSC of
S - S0) followed by batched top-k retrieval of the whole query batch.
`value` = queries per second of that step.  Beside it the JSON line reports
retrieval alone on a resident index (batched, and one query per launch with
p50/p99 latency), the build alone (docs/s), the end-to-end rate through the
host-buffer entry points, the roofline of the dominant kernel and the CPU
oracle's rate on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

from paper_2407_03618_gb300 import synth  # noqa: E402

L2_BYTES = 129 * 1024 * 1024


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="passage", choices=sorted(synth.WORKLOADS))
    p.add_argument("--variant", default="lucene", choices=list(synth.ALL_VARIANTS) + ["tfldp"])
    p.add_argument("--k", type=int, default=10)
    p.add_argument("--plain-queries", type=int, default=1000)
    p.add_argument("--cpu-sample-queries", type=int, default=32,
                   help="queries of the batch the oracle answers for cpu_baseline")
    p.add_argument("--ref-sample-queries", type=int, default=16,
                   help="queries per step of --impl reference")
    p.add_argument("--queries", type=int, default=0,
                   help="use only the first N queries of the batch (small profiler cases)")
    p.add_argument("--docs", type=int, default=0,
                   help="a corpus of N documents of the workload's law instead of its own size "
                        "(small profiler cases; the workload is then named <name>:<N>docs)")
    p.add_argument("--no-extras", action="store_true",
                   help="only the timed steps (used for profiler runs)")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the library's default plan instead of autotuning it")
    p.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    p.add_argument("--no-zipf1m", action="store_true",
                   help="skip the step measured on the 1M-document workload")
    return p.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ------------------------------------------------- ranks (weak scaling) ----
# Under torchrun every rank answers its own query batch over its own replica
# of the index; no data crosses ranks.  Only the timing is combined.

def rank_batch(w, rank: int, n_queries: int = 0):
    """The query batch of `rank`: the workload's query law with seed 1 + rank."""
    q = w.queries(seed=1 + rank)
    if n_queries:
        q = q.subset(np.arange(min(n_queries, q.n_queries)))
    return q


def max_over_ranks(ms: float, world: int, device) -> float:
    """The job's time: the slowest rank's (all_reduce MAX; a no-op at N = 1)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the job's time."""
    return units_per_rank * world / (ms / 1e3)


# ------------------------------------------------------------ clocks ------

class ClockSampler:
    """nvidia-smi samples (with their wall-clock timestamps) every 50 ms;
    stop() keeps those taken inside the window set by mark_start / mark_end,
    i.e. during the timed region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.t0 = self.t1 = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.5)  # let it start sampling before the timed region
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        import datetime
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    continue
                if self.t0 is not None and self.t1 is not None and not (self.t0 <= ts <= self.t1):
                    continue
                rows.append(parts[1:])
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------- CPU oracle -------

def oracle_rate(corpus, queries, variant, k, n_sample, threads, params):
    """The oracle (FP64 C, lazy exhaustive) as it stands, on a bounded sample:
    its build of the full corpus (1 thread, timed once), then top-k of
    n_sample evenly spaced queries of the batch on `threads` threads and of a
    few of them on one thread.  value = queries/s on all cores (the build is
    reported beside it, as docs/s, not folded in)."""
    import oracle
    t0 = time.perf_counter()
    orc = oracle.build(corpus.tokens, corpus.doc_offsets, corpus.vocab, oracle.VARIANTS[variant],
                       params["k1"], params["b"], params["delta"])
    t_build = time.perf_counter() - t0
    idx = np.linspace(0, queries.n_queries - 1, n_sample).astype(np.int64)
    sub = queries.subset(idx)
    t0 = time.perf_counter()
    oracle.topk(orc, sub.tokens, sub.offsets, k, n_threads=threads)
    t_all = time.perf_counter() - t0
    n1 = max(1, n_sample // 8)
    sub1 = queries.subset(idx[:n1])
    t0 = time.perf_counter()
    oracle.topk(orc, sub1.tokens, sub1.offsets, k, n_threads=1)
    t_1 = time.perf_counter() - t0
    return orc, {"value": n_sample / t_all, "unit": "queries/s", "cores": threads,
                 "kind": "oracle",
                 "sample": (f"lazy exhaustive top-{k} of {n_sample} evenly spaced queries of the "
                            f"batch on {threads} threads ({t_all:.2f} s) over the oracle's index "
                            f"of the full corpus; its build ({t_build:.1f} s, 1 thread) is "
                            f"reported as build_docs_per_s, not in value"),
                 "build_s": t_build, "build_docs_per_s": corpus.n_docs / t_build,
                 "ms_per_query": t_all / n_sample * 1e3,
                 "single_thread": {"value": n1 / t_1, "unit": "queries/s", "cores": 1,
                                   "queries": n1}}


def workload_of(args):
    """The workload to run: BASELINE-shaped as named, or (--docs N) the same
    laws over N documents for a small profiler case."""
    import dataclasses
    w = synth.WORKLOADS[args.workload]
    if args.docs:
        w = dataclasses.replace(w, name=f"{w.name}:{args.docs}docs", n_docs=args.docs)
    return w


def bench_config(args, w, n_queries: int, world: int) -> dict:
    """The `config` both arms print: the workload, the variant and k, and what
    one step of the GPU arm runs."""
    return {**w.describe(), "variant": args.variant, "k": args.k,
            "queries_per_step": n_queries,
            "step": "index build + batched top-k retrieval of the whole query batch",
            "l2": "inputs larger than L2 (no flush needed)",
            "parallelism": f"replicated index, {n_queries} queries per GPU, {world} GPU(s)"}


def reference_arm(args):
    """The oracle as it stands, on the host cores: its index is built once
    (timed, reported), then each step answers a bounded sample of the batch's
    queries (lazy exhaustive top-k on all cores).  value = queries answered /
    measured step time; the oracle's build is not in the step, which favours
    the oracle over the GPU arm (whose step includes its build)."""
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    w = workload_of(args)
    corpus = w.corpus()
    queries = rank_batch(w, 0, args.queries)
    threads = os.cpu_count() or 1
    import oracle
    t0 = time.perf_counter()
    orc = oracle.build(corpus.tokens, corpus.doc_offsets, corpus.vocab,
                       oracle.VARIANTS[args.variant], w.params["k1"], w.params["b"],
                       w.params["delta"])
    t_build = time.perf_counter() - t0
    n_sample = max(1, args.ref_sample_queries)
    rng = np.random.default_rng(7)
    times = []
    for step in range(args.warmup + args.steps):
        idx = rng.integers(0, queries.n_queries, n_sample)
        sub = queries.subset(idx)
        t0 = time.perf_counter()
        oracle.topk(orc, sub.tokens, sub.offsets, args.k, n_threads=threads)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    step_s = sum(times) / len(times)
    value = n_sample / step_s
    line = {"impl": "reference", "metric": f"queries/s @k={args.k}", "value": value,
            "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, w, queries.n_queries, world),
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": threads,
                             "kind": "oracle",
                             "sample": (f"each step = lazy exhaustive top-{args.k} of {n_sample} "
                                        f"random queries of the batch on {threads} threads over "
                                        f"the oracle's index of the full corpus (built once "
                                        f"before the steps in {t_build:.1f} s on 1 thread, not "
                                        f"in the step)"),
                             "build_s": t_build},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ GPU arm -----

def plan_key(plan):
    """A plan dict as the "plan:" line of a traffic file writes it."""
    return ",".join(str(plan[f]) for f in ("accumulator", "tile_docs", "block_threads",
                                           "dense_max_postings", "stage_entries", "stages")
                    if f in plan)


def parse_traffic(text, stamp, workload, plan):
    """DRAM bytes per launch from the "key: value" lines of a traffic profile
    (one ncu capture), or None.  The figure holds only for the code it was
    taken on (code_stamp: build_ext.code_stamp()), its workload and, when the
    profile names one, its plan."""
    kv = {}
    for line in text.splitlines():
        if ":" in line and not line.startswith("#"):
            key, _, val = line.partition(":")
            kv[key.strip().strip("`* ")] = val.strip().strip("`* ")
    try:
        if (kv.get("code_stamp") == stamp and kv.get("workload") == workload
                and kv.get("plan", plan) == plan):
            return int(kv["traffic_bytes_per_launch"])
    except (ValueError, KeyError):
        pass
    return None


def read_traffic(path, stamp, workload, plan):
    """parse_traffic of the file profiles/<kernel>_<workload>_traffic.md;
    None when there is no such file."""
    try:
        with open(path) as f:
            return parse_traffic(f.read(), stamp, workload, plan)
    except OSError:
        return None


def kernel_bytes(name, ctx, launches_per_step=1.0):
    """Algorithmic bytes per launch of the kernels a roofline is quoted for.
    The retrieval kernels' bytes are those of the whole batch, which a call
    splits into launches_per_step sub-batches when the tile candidates of
    all its queries do not fit the candidate budget."""
    if name == "k_tile_staged":
        return ctx["tile_bytes"] / max(launches_per_step, 1.0)
    if name == "k_dense_topk":
        return ctx["dense_bytes"] / max(launches_per_step, 1.0)
    if name == "k_radix_downsweep":
        return 16 * ctx["n_tokens"]  # read key + doc, write key + doc, 4 B each
    if name == "k_radix_upsweep":
        return 4 * ctx["n_tokens"]
    if name == "k_score":
        return 20 * ctx["nnz"]  # run start x2, term, doc in; tf, score out (4 B each)
    return None


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_03618_gb300 import bm25

    w = workload_of(args)
    prm = w.params
    corpus = w.corpus()
    queries = rank_batch(w, rank, args.queries)  # each rank its own batch (weak scaling)
    k = args.k
    nq = queries.n_queries

    tok = torch.from_numpy(corpus.tokens).to(dev)
    off = torch.from_numpy(corpus.doc_offsets).to(dev)
    qt = torch.from_numpy(queries.tokens).to(dev)
    qo = torch.from_numpy(queries.offsets).to(dev)
    ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
    sc = torch.empty((nq, k), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # the retrieval plan: autotuned once on this batch (a resident index),
    # then set on the index each step builds
    tuned = None
    if not args.no_autotune:
        ixt = bm25.Index.build(tok, off, corpus.vocab, args.variant, prm["k1"], prm["b"],
                               prm["delta"])
        tuned = ixt.autotune(qt, qo, k)
        ixt.close()
    plan = tuned[0] if tuned else None

    # retrieval scratch sized once for this batch and plan and reused by every
    # step (as a serving process keeps it), so no step allocates device memory
    # outside the index itself
    ix0 = bm25.Index.build(tok, off, corpus.vocab, args.variant, prm["k1"], prm["b"],
                           prm["delta"])
    ws = bm25.Workspace(ix0, nq, qt.numel(), k)
    ws.reserve(ix0, nq, qt.numel(), k, plan=plan)
    ix0.close()

    def step():
        ix = bm25.Index.build(tok, off, corpus.vocab, args.variant, prm["k1"], prm["b"],
                              prm["delta"])
        ix.retrieve(qt, qo, k, out=(ids, sc), workspace=ws, plan=plan)
        ix.close()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local)
    clocks = ClockSampler(gpu_id) if rank == 0 else None
    launches0 = bm25.launch_count()
    # (kernel launches before the timed region, for lining up a profiler's launch list)
    print(f"bench: {launches0} library kernel launches before the timed region",
          file=sys.stderr, flush=True)
    bm25.profile_begin()
    barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.mark_start()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if clocks:
        clocks.mark_end()
    barrier()
    prof = bm25.profile_end()
    launches = bm25.launch_count() - launches0
    clock_info = clocks.stop() if clocks else None
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    value = job_rate(nq, world, ms)

    line = {"metric": f"queries/s @k={k}", "value": value, "unit": "queries/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(args, w, nq, world),
            "clocks": clock_info, "gpu_launches": launches * world}
    if tuned:
        line["plan"] = {"chosen": tuned[0], "ms": tuned[1],
                        "tried": [{"plan": p_, "ms": m_} for p_, m_ in tuned[2]]}

    if not args.no_extras and rank == 0:
        extras(args, line, bm25, corpus, queries, tok, off, qt, qo, ids, sc, dev, prof, w, plan)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def extras(args, line, bm25, corpus, queries, tok, off, qt, qo, ids, sc, dev, prof, w, plan):
    import torch
    prm = w.params
    k = args.k
    nq = queries.n_queries
    stream = torch.cuda.current_stream(dev)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    ix = bm25.Index.build(tok, off, corpus.vocab, args.variant, prm["k1"], prm["b"], prm["delta"])
    if plan:
        ix.set_plan(**plan)
    used = ix.get_plan()
    info = ix.info()
    ex_indptr = ix.export(["indptr"])["indptr"]
    df = np.diff(ex_indptr)
    qlen = np.diff(queries.offsets)
    postings = int(df[queries.tokens].sum())
    retrieval_bytes = 8 * postings + 20 * int(qlen.sum()) + 8 * k * nq
    # per-query algorithmic bytes (postings, indptr pair and token, output),
    # split the way the library routes queries: at most dense_max postings ->
    # dense path, the rest tiled
    cs = np.concatenate([[0], np.cumsum(df[queries.tokens], dtype=np.int64)])
    qpost = cs[queries.offsets[1:]] - cs[queries.offsets[:-1]]
    qbytes = 8 * qpost + 20 * qlen + 8 * k
    dense_on = used["accumulator"] in (bm25.ACC_AUTO, bm25.ACC_L2_DENSE)
    dmax = used["dense_max_postings"] if used["accumulator"] == bm25.ACC_AUTO else \
        max(used["dense_max_postings"], 1 << 19)
    is_dense = (qpost <= dmax) if dense_on else np.zeros(nq, bool)
    ctx = {"retrieval_bytes": retrieval_bytes, "tile_bytes": int(qbytes[~is_dense].sum()),
           "dense_bytes": int(qbytes[is_dense].sum()), "n_tokens": corpus.n_tokens,
           "nnz": info["nnz"]}
    line["routing"] = {"plan": used, "dense_queries": int(is_dense.sum()),
                       "tiled_queries": int((~is_dense).sum()),
                       "dense_postings_frac": float(qpost[is_dense].sum() / max(1, qpost.sum()))}

    # kernel shares over the timed region
    total_ms = sum(v[1] for v in prof.values()) or 1.0
    kernels = {n: {"launches": c, "ms_per_launch": t / max(c, 1), "share": t / total_ms}
               for n, (c, t) in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    line["kernels"] = kernels
    top = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None

    def roofline_for(name, c, t):
        b = kernel_bytes(name, ctx, c / max(args.steps, 1))
        if b is None:
            return None
        avg_s = t / c / 1e3
        achieved = b / avg_s / 1e9
        from paper_2407_03618_gb300 import build_ext
        traffic = read_traffic(os.path.join(ROOT, "profiles",
                                            f"{name}_{w.name.replace('-', '')}_traffic.md"),
                               build_ext.code_stamp(), w.name, plan_key(used))
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": traffic,
                "algorithmic_bytes_per_launch": b, "ms_per_launch": t / c,
                "peak_source": f"{peak_src} hbm_gbs (STREAM-style copy)"}

    if top is not None:
        c, t = prof[top]
        line["roofline"] = roofline_for(top, c, t)
        if line["roofline"] is None:
            line["roofline"] = {"kernel": top, "bound": "hbm", "achieved": None,
                                "peak": hbm_peak, "unit": "GB/s", "frac": None, "traffic": None}
        others = {}
        for n in ("k_tile_staged", "k_dense_topk", "k_radix_downsweep"):
            if n in prof and n != top:
                others[n] = roofline_for(n, *prof[n])
        line["roofline_other"] = others

    # retrieval alone on the resident index, batched (k and 100)
    def time_retrieval(kk, reps=10):
        o = (torch.empty((nq, kk), dtype=torch.int32, device=dev),
             torch.empty((nq, kk), dtype=torch.float32, device=dev))
        for _ in range(3):
            ix.retrieve(qt, qo, kk, out=o)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            ix.retrieve(qt, qo, kk, out=o)
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    r_ms = time_retrieval(k)
    r100_ms = time_retrieval(100)
    line["retrieval"] = {"qps": nq / (r_ms / 1e3), "ms_per_batch": r_ms,
                         "qps_k100": nq / (r100_ms / 1e3), "ms_per_batch_k100": r100_ms,
                         "postings_per_query": postings / nq,
                         "algorithmic_GBps": retrieval_bytes / (r_ms / 1e3) / 1e9,
                         "hbm_frac": retrieval_bytes / (r_ms / 1e3) / 1e9 / hbm_peak}

    # plain path: one query per launch, untuned, latency per query
    P = min(args.plain_queries, nq)
    singles = []
    for i in range(P):
        a0, a1 = int(queries.offsets[i]), int(queries.offsets[i + 1])
        singles.append((qt[a0:a1].clone(),
                        torch.tensor([0, a1 - a0], dtype=torch.int64, device=dev)))
    o1 = (torch.empty((1, k), dtype=torch.int32, device=dev),
          torch.empty((1, k), dtype=torch.float32, device=dev))
    for i in range(min(20, P)):
        ix.retrieve(singles[i][0], singles[i][1], k, out=o1)
    torch.cuda.synchronize(dev)
    lat = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(P)]
    t0 = time.perf_counter()
    for i in range(P):
        ev[i][0].record(stream)
        ix.retrieve(singles[i][0], singles[i][1], k, out=o1)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    lat = sorted(e[0].elapsed_time(e[1]) for e in ev)
    line["plain_path"] = {"queries": P, "qps": P / wall,
                          "p50_ms": lat[len(lat) // 2], "p99_ms": lat[int(0.99 * (len(lat) - 1))],
                          "batched_speedup": (nq / (r_ms / 1e3)) / (P / wall)}
    # the same one-query calls through the host-buffer entry point (query in,
    # result out of host memory): comparable with served latency
    hl = []
    hq = [(queries.query(i).astype(np.int32), np.array([0, queries.query(i).shape[0]], np.int64))
          for i in range(min(P, 300))]
    hout = (np.zeros((1, k), np.int32), np.zeros((1, k), np.float32))
    for t_, o_ in hq[:10]:
        ix.retrieve_host(t_, o_, k, out=hout)
    t0 = time.perf_counter()
    for t_, o_ in hq:
        a_ = time.perf_counter()
        ix.retrieve_host(t_, o_, k, out=hout)
        hl.append((time.perf_counter() - a_) * 1e3)
    hwall = time.perf_counter() - t0
    hl.sort()
    line["plain_path"]["host"] = {"queries": len(hq), "qps": len(hq) / hwall,
                                  "p50_ms": hl[len(hl) // 2],
                                  "p99_ms": hl[int(0.99 * (len(hl) - 1))]}
    line["batched_latency_ms"] = {"p50": r_ms, "p99": r_ms,
                                  "note": "every query of a batch completes with the batch"}

    # index build alone
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ix.close()
    torch.cuda.synchronize(dev)
    a.record(stream)
    for _ in range(3):
        bm25.Index.build(tok, off, corpus.vocab, args.variant, prm["k1"], prm["b"],
                         prm["delta"]).close()
    b.record(stream)
    torch.cuda.synchronize(dev)
    b_ms = a.elapsed_time(b) / 3
    build_bytes = (4 * corpus.n_tokens + 8 * (corpus.n_docs + 1) + 8 * info["nnz"]
                   + 8 * (corpus.vocab + 1) + 16 * corpus.vocab)
    line["index_build"] = {"ms": b_ms, "docs_per_s": corpus.n_docs / (b_ms / 1e3),
                           "nnz": info["nnz"], "n_tokens": corpus.n_tokens,
                           "algorithmic_GBps": build_bytes / (b_ms / 1e3) / 1e9}

    # end to end through the host-buffer entry points (pinned host memory)
    h_tok = torch.from_numpy(corpus.tokens).pin_memory()
    h_off = torch.from_numpy(corpus.doc_offsets).pin_memory()
    h_qt = torch.from_numpy(queries.tokens).pin_memory()
    h_qo = torch.from_numpy(queries.offsets).pin_memory()
    h_ids = torch.empty((nq, k), dtype=torch.int32).pin_memory()
    h_sc = torch.empty((nq, k), dtype=torch.float32).pin_memory()

    phases = []

    def e2e_step():
        t_a = time.perf_counter()
        ih = bm25.Index.build_host(h_tok, h_off, corpus.vocab, args.variant, prm["k1"], prm["b"],
                                   prm["delta"])
        t_b = time.perf_counter()
        ih.retrieve_host(h_qt, h_qo, k, out=(h_ids, h_sc))
        t_c = time.perf_counter()
        ih.close()
        phases.append((t_b - t_a, t_c - t_b, time.perf_counter() - t_c))

    e2e_step()
    phases.clear()
    steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / steps
    h2d = 4 * corpus.n_tokens + 8 * (corpus.n_docs + 1) + 4 * queries.tokens.shape[0] + 8 * (nq + 1)
    med = np.median(np.array(phases), axis=0) * 1e3
    line["e2e"] = {"value": nq / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": 8 * nq * k, "ms_per_step": e2e_s * 1e3,
                   "median_ms": {"build_host": float(med[0]), "retrieve_host": float(med[1]),
                                 "close": float(med[2])}}

    if not args.no_serving:
        line["serving"] = serving(args, bm25, corpus, queries, tok, off, dev, w, plan,
                                  line["plain_path"])

    if w.name != "zipf-1m" and not args.no_zipf1m:
        line["zipf1m"] = other_workload_step(args, bm25, dev, "1m", hbm_peak)

    # CPU oracle on a bounded sample (rank 0, N = 1 only)
    if line["n_gpus"] == 1:
        _, cpu = oracle_rate(corpus, queries, args.variant, k, args.cpu_sample_queries,
                             os.cpu_count() or 1, prm)
        line["cpu_baseline"] = cpu


def other_workload_step(args, bm25, dev, name, hbm_peak):
    """The same step (build + batched retrieval of the whole batch at k) on
    another workload, its plan autotuned on its own batch."""
    import torch
    w = synth.WORKLOADS[name]
    prm = w.params
    c, q = w.corpus(), w.queries()
    tok = torch.from_numpy(c.tokens).to(dev)
    off = torch.from_numpy(c.doc_offsets).to(dev)
    qt = torch.from_numpy(q.tokens).to(dev)
    qo = torch.from_numpy(q.offsets).to(dev)
    k = args.k
    ix = bm25.Index.build(tok, off, c.vocab, args.variant, prm["k1"], prm["b"], prm["delta"])
    plan = ix.autotune(qt, qo, k)[0]
    ws = bm25.Workspace(ix, q.n_queries, qt.numel(), k)
    ws.reserve(ix, q.n_queries, qt.numel(), k, plan=plan)
    df = np.diff(ix.export(["indptr"])["indptr"])
    ix.close()
    out = (torch.empty((q.n_queries, k), dtype=torch.int32, device=dev),
           torch.empty((q.n_queries, k), dtype=torch.float32, device=dev))

    def step():
        i2 = bm25.Index.build(tok, off, c.vocab, args.variant, prm["k1"], prm["b"], prm["delta"])
        i2.retrieve(qt, qo, k, out=out, workspace=ws, plan=plan)
        i2.close()

    for _ in range(3):
        step()
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    bm25.profile_begin()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 10
    a.record(stream)
    for _ in range(n):
        step()
    b.record(stream)
    torch.cuda.synchronize(dev)
    prof = bm25.profile_end()
    ms = a.elapsed_time(b) / n
    postings = int(df[q.tokens].sum())
    res = {"workload": w.name, "queries_per_step": q.n_queries, "ms_per_step": ms,
           "value": q.n_queries / (ms / 1e3), "unit": "queries/s", "plan": plan,
           "postings_per_query": postings / q.n_queries}
    if "k_tile_staged" in prof:
        cnt, t = prof["k_tile_staged"]
        res["k_tile_staged_ms"] = t / cnt
    ws.close()
    return res


def serving(args, bm25, corpus, queries, tok, off, dev, w, plan, plain):
    """Requests one query at a time with Poisson arrivals over eight resident
    indexes (the batch's corpus and seven smaller ones of the other workload
    shapes), k drawn from {10, 100, 1000}, through the library's
    continuous-batching server.  Latency = submit to result, measured by the
    server; compared with the one-query-per-launch path (plain_path)."""
    import torch
    prm = w.params
    shapes = [  # (docs, vocab, zipf s, length law): the tiny, 1M and passage shapes, scaled
        (10_000, 5_000, 1.1, ("poisson", 60)), (25_000, 20_000, 1.05, ("lognormal", 60, 0.6)),
        (50_000, 50_000, 1.0, ("lognormal", 56, 0.5)), (100_000, 5_000, 1.1, ("poisson", 60)),
        (200_000, 100_000, 1.05, ("lognormal", 60, 0.6)),
        (400_000, 200_000, 1.0, ("lognormal", 56, 0.5)),
        (150_000, 50_000, 1.1, ("poisson", 30))]
    idx, vocabs = [], []
    ix0 = bm25.Index.build(tok, off, corpus.vocab, args.variant, prm["k1"], prm["b"], prm["delta"])
    if plan:
        ix0.set_plan(**plan)
    idx.append(ix0)
    vocabs.append(corpus.vocab)
    for i, (n, v, s_, L) in enumerate(shapes):
        c = synth.make_corpus(n, v, s_, L, seed=100 + i)
        idx.append(bm25.Index.build(torch.from_numpy(c.tokens).to(dev),
                                    torch.from_numpy(c.doc_offsets).to(dev), c.vocab,
                                    args.variant, prm["k1"], prm["b"], prm["delta"]))
        vocabs.append(c.vocab)
    rng = np.random.default_rng(11)
    out = {"indexes": [ix.info()["n_docs"] for ix in idx], "rates": []}
    srv = bm25.Server(idx, max_batch_queries=2048, max_inflight=3, k_max=1000)
    for rate, n_req in ((5_000, 5_000), (20_000, 20_000), (50_000, 40_000)):
        which = rng.integers(0, len(idx), n_req)
        lens = rng.integers(1, 33, n_req)
        ks = rng.choice([10, 100, 1000], n_req)
        reqs = []
        for i in range(n_req):
            if which[i] == 0:  # a query of the batch's own workload
                reqs.append(queries.query(int(rng.integers(0, queries.n_queries))))
            else:
                reqs.append(synth.zipf_sampler(vocabs[which[i]], 1.05)(rng, int(lens[i])))
        arrival = np.cumsum(rng.exponential(1.0 / rate, n_req))
        srv.stats(reset=True)
        t0 = time.perf_counter()
        tickets = srv.replay(which, reqs, ks, arrival)  # submitted natively at their times
        t_sub = time.perf_counter() - t0
        for i, tk in enumerate(tickets):
            srv.poll(tk, int(ks[i]))
        st = srv.stats()
        # the same requests at the same arrival times through the plain path:
        # one query per call (host buffers in and out), served in order
        t0 = time.perf_counter()
        plain_lat = np.sort(bm25.replay_plain(idx, which, reqs, ks, arrival)) / 1e3
        p_span = time.perf_counter() - t0
        out["rates"].append({"offered_qps": rate, "requests": n_req,
                             "submit_s": t_sub, "arrivals_s": float(arrival[-1]),
                             "achieved_qps": st["completed"] / max(st["span_us"] / 1e6, 1e-9),
                             "span_s": st["span_us"] / 1e6,
                             "p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3,
                             "max_ms": st["max_us"] / 1e3,
                             "mean_batch": st["batched_queries"] / max(1, st["batches"]),
                             "failed": st["failed"],
                             "plain_same_arrivals": {
                                 "achieved_qps": n_req / p_span,
                                 "p50_ms": float(plain_lat[len(plain_lat) // 2]),
                                 "p99_ms": float(plain_lat[int(0.99 * (len(plain_lat) - 1))]),
                                 "max_ms": float(plain_lat[-1])}})
    srv.close()
    for ix in idx:
        ix.close()
    out["plain_path_host"] = plain.get("host")
    out["note"] = ("requests submitted at their Poisson arrival times by a native loop "
                   "(bm25_server_replay); achieved_qps = completed / (first submit .. last "
                   "completion, recorded by the server); latency = submit to result on the host.  "
                   "plain_same_arrivals: the same requests at the same arrival times through the "
                   "one-query-per-call host entry point, served in order natively "
                   "(bm25_replay_plain; latency = arrival to result).  plain_path_host: that "
                   "entry point back to back, no queueing")
    return out


if __name__ == "__main__":
    sys.exit(main())
