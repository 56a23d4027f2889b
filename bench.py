#!/usr/bin/env python3
"""Benchmark: exact sparse spherical k-means, whole clustering jobs on synthetic tf-idf data.

One step = one complete clustering job (skm_fit): the Lloyd loop of the paper (Sec. 2)
from k seeded initial documents, with the non-changing-clusters skip (Sec. 3.1), BF16
centroids scored with FP32 accumulation, FP64 rescoring of near ties, and the
deterministic centroid update, up to the workload's iteration limit or until no
assignment changes. Every assignment step, update and objective runs on the GPU.

Metric: documents assigned per second per iteration (N x iterations / time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload large|medium|small]
  python bench.py --impl reference ...   (the FP64 CPU oracle on host cores)

Variants of a fit workload for comparisons and profiling (the JSON config records them):
  --precision bf16|fp32  --prune ncc|none|ncc_index  --rescore on|off  --max-iter N
  --sparse-div D (sparse centroid rows)  --case N,D,K (documents, vocabulary, clusters)  --k K

Under torchrun (N > 1) each rank runs an independent replica (different seeds) on its
own GPU; the job value is the sum of the ranks' documents over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# DRAM bytes (read + write) of one k_score launch of the large workload's first step (a
# full pass: 2M documents x 10,000 centroids, 325 ms), from one ncu capture recorded in
# profiles/k_score_traffic_large_full_pass.md; it is reported for the default large
# workload only and must be retaken whenever k_score changes.
LARGE_FULL_PASS_TRAFFIC = 951.08e9 + 1.29e9
LARGE_FULL_PASS_ALG_BYTES = 7.43e9
LARGE_FULL_PASS_SCOPE = ("one full-pass k_score launch of step 1 (2M documents x 10,000 centroids, all nonzeros "
                         f"gathered); algorithmic bytes of that launch {LARGE_FULL_PASS_ALG_BYTES:.3g}")

# With the head on the tensor cores (the default), one full pass of the first step is 20
# chunks of k_head_rows + k_head_gemm + k_score over the tail nonzeros; DRAM bytes of the 20
# launches of each, from the capture in the same profile (second section).
LARGE_HEAD_FULL_PASS_TRAFFIC = {"k_score (tail)": 930.4e9 + 1.3e9, "k_head_gemm": 4.8e9 + 39.8e9,
                                "k_head_rows": 1.0e9 + 2.9e9}
LARGE_HEAD_FULL_PASS_SCOPE = ("one full pass of step 1 (2M documents x 10,000 centroids), 20 launches of each kernel; "
                              f"algorithmic bytes of the pass {LARGE_FULL_PASS_ALG_BYTES:.3g}")

METRIC = "docs assigned/s per iteration"
UNIT = "docs/s"
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def device_sm_count(local: int = 0) -> int:
    """Streaming multiprocessors of the device the benchmark runs on (152 on a GB300)."""
    import torch
    return int(torch.cuda.get_device_properties(local).multi_processor_count)


def peaks(n_sm: int) -> dict:
    p = {"hbm_gbs": 6800.0, "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            m = json.load(f)
        p = {"hbm_gbs": float(m["hbm_gbs"]), "source": "measured",
             "sm_max_mhz": float(m.get("sm_max_mhz", SM_MAX_MHZ))}
    # FP32 FMA peak from unit counts and the maximum SM clock: SMs (read from the device) x
    # 128 FP32 lanes x 2 flop
    mhz = p.get("sm_max_mhz", SM_MAX_MHZ)
    p["n_sm"] = n_sm
    p["fp32_tflops"] = n_sm * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    p["fp32_source"] = (f"FP32 FMA: {n_sm} SMs (device multiProcessorCount) x {FP32_LANES_PER_SM} lanes x "
                        f"2 flop x {mhz:g} MHz (derived)")
    return p


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ distributed
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        import torch
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x: float, device) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x: float, device) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle legs
def oracle_sample_rate(docs, C32: np.ndarray, seed: int, budget_s: float = 15.0):
    """The FP64 oracle's assignment step (plain definition, Sec. 2) on a bounded, seeded
    sample of the workload's documents: returns (docs/s, sample size, seconds, threads)."""
    import oracle
    from paper_2108_00895_gb300 import synth
    # calibrate on growing probes until one takes at least 0.5 s, then size the sample
    n_probe, per_doc = 64, None
    while True:
        probe = docs.rows(synth.sample_ids(docs.n_docs, n_probe, seed))
        t0 = time.perf_counter()
        oracle.assign(probe, C32)
        dt = time.perf_counter() - t0
        per_doc = max(dt / probe.n_docs, 1e-8)
        if dt >= 0.5 or n_probe >= docs.n_docs:
            break
        n_probe = min(docs.n_docs, n_probe * 4)
    n = int(min(docs.n_docs, max(64, budget_s / per_doc)))
    sample = docs.rows(synth.sample_ids(docs.n_docs, n, seed + 1))
    t0 = time.perf_counter()
    oracle.assign(sample, C32)
    dt = time.perf_counter() - t0
    return n / dt, n, dt, oracle.num_threads()


def oracle_modes(docs, w, seed: int, n_sample: int = 20000, max_iter: int = 10):
    """The paper's three CPU methods (Sec. 4.1-4.2, Table 1) as the oracle restates them --
    Baseline (plain Lloyd), NCC (Sec. 3.1) and NCC+INDEX (Sec. 3.2, thresholds of Sec. 4.1) --
    each a complete fit of a bounded seeded sample of the workload (n_sample documents, the
    workload's vocabulary, k = n_sample / 200 clusters: the large workload's 200 documents per
    cluster), with every host core and with one thread."""
    import oracle
    from paper_2108_00895_gb300 import synth
    n = min(n_sample, docs.n_docs)
    sample = docs.rows(synth.sample_ids(docs.n_docs, n, seed))
    k = max(2, min(w.k, n // 200))
    ids = synth.init_ids(n, k, seed + 1)
    all_cores = oracle.num_threads()
    out = {"sample": f"{n} seeded documents of the workload, k = {k}, at most {max_iter} steps, "
                     f"stop on unchanged assignments", "cores_all": all_cores, "modes": {}}
    try:
        for threads in (all_cores, 1):
            oracle.set_threads(threads)
            for mode in ("plain", "ncc", "ncc_index"):
                t0 = time.perf_counter()
                r = oracle.fit(sample, k, ids, max_iter, mode=mode)
                dt = time.perf_counter() - t0
                out["modes"].setdefault(mode, {})[f"threads_{threads}"] = {
                    "docs_per_s_per_iter": n * r.iters / dt, "seconds": dt, "iters": r.iters,
                    "sims": int(r.sims.sum())}
    finally:
        oracle.set_threads(all_cores)
    return out


def run_reference(args, w, world, rank, dist):
    """Reference arm: the FP64 oracle as it stands, timed on the host cores."""
    if rank != 0:
        return
    import oracle
    from paper_2108_00895_gb300 import synth
    docs = w.corpus()
    ids = w.init_ids()
    # c_j = x_{init_j}, stored as float32 (the oracle widens it exactly) to halve host memory
    C0 = np.zeros((docs.n_terms, w.k), np.float32)
    for j, i in enumerate(ids):
        a, b = docs.row_ptr[i], docs.row_ptr[i + 1]
        C0[docs.col_idx[a:b], j] = docs.values[a:b]
    # size one step's sample so that warmup + steps stay within a few minutes
    n_probe = 32
    while True:
        probe = docs.rows(synth.sample_ids(docs.n_docs, n_probe, 7))
        t0 = time.perf_counter()
        oracle.assign(probe, C0)
        dt = time.perf_counter() - t0
        per_doc = max(dt / probe.n_docs, 1e-8)
        if dt >= 0.5 or n_probe >= docs.n_docs:
            break
        n_probe = min(docs.n_docs, n_probe * 4)
    total_budget = 150.0
    n = int(min(docs.n_docs, max(32, total_budget / (args.steps + args.warmup) / per_doc)))
    times = []
    for s in range(args.warmup + args.steps):
        sample = docs.rows(synth.sample_ids(docs.n_docs, n, 100 + s))
        t0 = time.perf_counter()
        oracle.assign(sample, C0)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = n / (sum(times) / len(times))
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(w.describe(), sample_docs_per_step=n, centroids="initial documents"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} seeded documents of the workload per step, assignment "
                                       f"step against the k initial centroids"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workloads_large_name() -> str:
    from paper_2108_00895_gb300 import workloads
    return workloads.LARGE.name


# ------------------------------------------------------------------ our arm
def run_ours(args, w, world, rank, local, dist):
    import torch

    from paper_2108_00895_gb300 import skm

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    skm.load()
    if rank != 0:
        w = w.scaled(seed_id=w.seed_id + 100 * rank)
    docs = w.corpus()
    ids = w.init_ids()
    N = docs.n_docs
    d_docs = (torch.from_numpy(docs.row_ptr).to(dev), torch.from_numpy(docs.col_idx).to(dev),
              torch.from_numpy(docs.values).to(dev))
    stream = torch.cuda.current_stream(dev)
    km = skm.SphericalKMeans(w.k, precision=w.precision, prune=w.prune, max_iter=w.max_iter,
                             shift_tol=w.shift_tol, rescore=args.rescore == "on", tau=args.tau, device=local,
                             stream=stream.cuda_stream, timing=True, sparse_div=args.sparse_div,
                             index_min_changed=args.index_min_changed, index_max_cands=args.index_max_cands,
                             head_terms=args.head_terms)
    a_dev = torch.empty(N, dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        km.fit(d_docs, ids, n_terms=docs.n_terms, assign_out=a_dev)
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    iters = 0
    agg = {"fmas": 0, "fmas_exec": 0, "bytes": 0, "ms_score": 0.0, "ms_decide": 0.0, "ms_update": 0.0,
           "launches_total": 0, "launches_score": 0, "sims": 0, "docs_pruned": 0, "docs_full": 0,
           "docs_rescored": 0, "docs_rescored_full": 0, "index_docs": 0, "index_sims": 0, "index_entries": 0,
           "index_products": 0, "ms_query": 0.0, "ms_index": 0.0, "ms_head": 0.0, "nnz_head": 0}
    objectives = None
    for _ in range(args.steps):
        r = km.fit(d_docs, ids, n_terms=docs.n_terms, assign_out=a_dev)
        iters += r.iters
        objectives = r.objective
        for key in agg:
            agg[key] += r.stats[key]
        agg["head_terms"] = r.stats["head_terms"]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(dist)
    clk = clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    t_max = max_over_ranks(dist, elapsed_ms, dev)
    docs_done = sum_over_ranks(dist, float(N * iters), dev)
    value = docs_done / (t_max / 1e3)

    # end to end through the public API with host buffers: the CSR and the assignment live in
    # pinned host memory, so that the library's copies run at DMA speed
    e2e = None
    if not args.no_e2e:
        from paper_2108_00895_gb300 import synth

        def pinned(x):
            return torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()

        docs_h = synth.Csr(pinned(docs.row_ptr), pinned(docs.col_idx), pinned(docs.values), docs.n_terms)
        a_host = torch.empty(N, dtype=torch.int32).pin_memory().numpy()
        barrier(dist)
        t0 = time.perf_counter()
        e_iters = 0
        for _ in range(args.steps):
            r = km.fit(docs_h, ids, assign_out=a_host)
            e_iters += r.iters
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dist, dt, dev)
        e_docs = sum_over_ranks(dist, float(N * e_iters), dev)
        e2e = {"value": e_docs / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(8 * (N + 1) + 8 * docs.nnz),
               "d2h_bytes_per_step": int(4 * N + 8 * (e_iters // max(args.steps, 1))),
               "host_memory": "pinned"}

    pk = peaks(device_sm_count(local))
    fl = 2.0 * agg["fmas_exec"]          # multiply-adds the scoring passes executed
    default_large = (w.name == workloads_large_name() and args.sparse_div == 0)
    # the scoring pass: the gather kernel over the tail nonzeros (or all of them) plus, when
    # the tensor-core head is on, its preparation and the head GEMM
    score_s = (agg["ms_score"] + agg["ms_head"]) / 1e3
    achieved_tf = fl / score_s / 1e12 if score_s > 0 else None
    hbm_gbs = agg["bytes"] / score_s / 1e9 if score_s > 0 else None
    t_roof = max(agg["bytes"] / (pk["hbm_gbs"] * 1e9), fl / (pk["fp32_tflops"] * 1e12))
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": pk["fp32_tflops"], "unit": "TFLOP/s",
                "frac": achieved_tf / pk["fp32_tflops"] if achieved_tf else None,
                "traffic": LARGE_FULL_PASS_TRAFFIC if default_large and not agg.get("head_terms") else None,
                "traffic_scope": LARGE_FULL_PASS_SCOPE if default_large and not agg.get("head_terms") else None,
                "traffic_full_pass": (dict(LARGE_HEAD_FULL_PASS_TRAFFIC, scope=LARGE_HEAD_FULL_PASS_SCOPE)
                                      if default_large and agg.get("head_terms") and args.head_terms == 0 else None),
                "kernel": ("scoring pass: k_head_gemm (tensor cores, the collection's most frequent terms) + "
                           "k_score (gathers over the other nonzeros, top-4 per slice)"
                           if agg.get("head_terms") else
                           "k_score (scoring pass: fused CSR x term-major centroid SpMM + top-4)"),
                "head": {"terms": agg.get("head_terms"), "ms_per_step": agg["ms_head"] / args.steps,
                         "nnz_share": agg["nnz_head"] / args.steps / docs.nnz if args.steps else None},
                "peak_source": pk["fp32_source"],
                "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": pk["hbm_gbs"],
                        "frac": hbm_gbs / pk["hbm_gbs"] if hbm_gbs else None,
                        "peak_source": f"{pk['source']} copy bandwidth"},
                "combined_frac": t_roof / score_s if score_s > 0 else None,
                "algorithmic": {"flop_per_step": fl / args.steps, "bytes_per_step": agg["bytes"] / args.steps,
                                "score_ms_per_step": agg["ms_score"] / args.steps,
                                "head_ms_per_step": agg["ms_head"] / args.steps,
                                "decide_ms_per_step": agg["ms_decide"] / args.steps,
                                "update_ms_per_step": agg["ms_update"] / args.steps,
                                "index_query_ms_per_step": agg["ms_query"] / args.steps,
                                "index_build_ms_per_step": agg["ms_index"] / args.steps,
                                "index_docs_per_step": agg["index_docs"] / args.steps}}

    cpu = None
    checks = {}
    C_fin = None
    if rank == 0 and world == 1 and not (args.no_cpu_baseline and args.no_checks):
        C_fin = km.centroids()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, n, dt, cores = oracle_sample_rate(docs, C_fin, 4242, args.cpu_budget)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} seeded documents of the workload, one assignment step (plain FP64 "
                         f"definition) against the final centroids, {dt:.1f} s",
               "paper_methods": oracle_modes(docs, w, 4343)}
    if rank == 0 and world == 1 and not args.no_checks:
        checks["error_vs_oracle"] = error_vs_oracle(skm, km, w, docs, ids, d_docs, a_dev, C_fin, objectives,
                                                    args, local, stream)
    del C_fin
    km.close()
    if rank == 0 and world == 1 and not args.no_checks:
        checks["speedup_vs_fp32_full"] = fp32_full_speedup(skm, w, docs, ids, d_docs, args, local, stream, value)
        if w.name == workloads_large_name() and args.serve_check_seconds > 0:
            from paper_2108_00895_gb300 import workloads
            checks["serving"] = serving_session(workloads.SERVING, local, args.serve_check_seconds, args.tau,
                                                job_slots=args.serve_job_slots)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if w.precision == "bf16" else "f32",
                "data": "synthetic",
                "config": dict(w.describe(), parallelism=f"replicas x{world}",
                               step="one full clustering job (fit)", iterations_per_step=iters / args.steps,
                               l2="inputs larger than L2 (CSR + centroid matrices >> 129 MB)",
                               objective_last=float(objectives[-1]) if objectives is not None else None,
                               tau=args.tau, rescore=args.rescore, sparse_div=args.sparse_div,
                               head_terms=agg.get("head_terms"),
                               index_min_changed=args.index_min_changed if w.prune == "ncc_index" else None,
                               index_max_cands=args.index_max_cands if w.prune == "ncc_index" else None),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": int(agg["launches_total"]),
                "work": {k_: v for k_, v in agg.items()}}
        line.update(checks)
        print(json.dumps(line), flush=True)


def error_vs_oracle(skm, km, w, docs, ids, d_docs, a_dev, C_fin, objectives, args, local, stream):
    """The timed job's results against the FP64 oracle (outside the timed region):
    - assignments of a seeded sample of documents against the final centroids (skm_assign):
      mismatches where the oracle's top-2 margin is at least 1e-5 (the contract: none), and
      in all;
    - the final update: sampled populated centroid columns against the oracle's normalised
      member sums of the job's final assignment (max-abs, FP32 master);
    - the last step's objective against the oracle's sum over all documents, computed with
      the centroids that step scored (a deterministic fit one step shorter gives them)."""
    import oracle
    from paper_2108_00895_gb300 import synth
    t0 = time.perf_counter()
    out = {}
    sample = docs.rows(synth.sample_ids(docs.n_docs, 4000, 4244))
    a_g, _ = km.assign(sample)
    a_or, s1, s2 = oracle.assign(sample, C_fin)
    clear = (s1 - s2) >= 1e-5
    out["assign_sample_docs"] = int(sample.n_docs)
    out["assign_mismatch_clear_margin"] = int(((a_g != a_or) & clear).sum())
    out["assign_mismatch_all"] = int((a_g != a_or).sum())
    out["assign_near_ties"] = int((~clear).sum())
    a_fin = a_dev.cpu().numpy()
    sizes = np.bincount(a_fin, minlength=w.k)
    pop = np.nonzero(sizes > 0)[0]
    cols = pop[synth.sample_ids(len(pop), min(40, len(pop)), 4245)]
    ref = oracle.centroids_subset(docs, a_fin, cols)
    out["centroid_max_abs"] = float(np.abs(C_fin[:, cols].astype(np.float64) - ref).max())
    out["centroid_columns"] = int(len(cols))
    T = len(objectives) if objectives is not None else 0
    if T > 1:
        with skm.SphericalKMeans(w.k, precision=w.precision, prune=w.prune, max_iter=T - 1, shift_tol=w.shift_tol,
                                 rescore=args.rescore == "on", tau=args.tau, device=local, stream=stream.cuda_stream,
                                 sparse_div=args.sparse_div, index_min_changed=args.index_min_changed,
                                 index_max_cands=args.index_max_cands, head_terms=args.head_terms) as k2:
            r2 = k2.fit(d_docs, ids, n_terms=docs.n_terms)
            C_prev = k2.centroids() if r2.iters == T - 1 else None
        if C_prev is not None:
            obj = oracle.objective(docs, C_prev, a_fin)
            out["objective_rel_err"] = float(abs(float(objectives[-1]) - obj) / abs(obj))
            out["objective_step"] = T
        del C_prev
    out["contract"] = "assignments exact where margin >= 1e-5; objective 1e-6 relative; centroids 1e-5 max-abs"
    out["seconds"] = time.perf_counter() - t0
    return out


def fp32_full_speedup(skm, w, docs, ids, d_docs, args, local, stream, value):
    """The plain FP32 full-comparison path on the same corpus (FP32 centroids, no pruning, no
    rescoring), a few steps after one warm-up fit, timed with CUDA events on the stream: its
    documents assigned per second per iteration, and the timed job's value over it."""
    import torch
    n_it = 3
    with skm.SphericalKMeans(w.k, precision="fp32", prune="none", max_iter=n_it, shift_tol=-1.0, rescore=False,
                             tau=args.tau, device=local, stream=stream.cuda_stream) as kf:
        kf.fit(d_docs, ids, n_terms=docs.n_terms)
        torch.cuda.synchronize(local)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = kf.fit(d_docs, ids, n_terms=docs.n_terms)
        e1.record(stream)
        torch.cuda.synchronize(local)
        ms = e0.elapsed_time(e1)
    rate = docs.n_docs * r.iters / (ms / 1e3)
    return {"fp32_full_docs_per_s_per_iter": rate, "steps": int(r.iters), "ms": ms,
            "speedup": value / rate,
            "path": "FP32 centroids, no pruning, no rescoring; the first steps of a fit from the same documents"}


# ------------------------------------------------------------------ batched form
def run_batched(args, world, rank, local, dist):
    """Batched form: all instances of the batched workload in one skm_fit_batched call per step
    (persistent scoring launch over all instances, loop captured in a CUDA graph)."""
    import tempfile

    import torch

    from paper_2108_00895_gb300 import skm, workloads
    W = workloads.BATCHED
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    skm.load()
    inst = W.instances()
    n_total = sum(d.n_docs for d, _, _ in inst)
    dinst = [((torch.from_numpy(d.row_ptr).to(dev), torch.from_numpy(d.col_idx).to(dev),
               torch.from_numpy(d.values).to(dev), d.n_terms), k, ids) for d, k, ids in inst]
    cache = os.path.join(tempfile.gettempdir(), f"skm_tune_{os.getpid()}.txt")
    for _ in range(args.warmup):
        skm.fit_batched(dinst, W.max_iter, tau=args.tau, use_graph=True, tune_cache=cache, device=local)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(dist)
    t0 = time.perf_counter()
    loop_ms, fmas, st = 0.0, 0, None
    for _ in range(args.steps):
        _, st = skm.fit_batched(dinst, W.max_iter, tau=args.tau, use_graph=True, tune_cache=cache, device=local)
        loop_ms += st["ms_loop"]
        fmas += st["fmas"]
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    barrier(dist)
    clk = clocks.stop()
    t_max = max_over_ranks(dist, dt, dev)
    docs_done = sum_over_ranks(dist, float(n_total * W.max_iter * args.steps), dev)
    e2e = None
    if not args.no_e2e:
        from paper_2108_00895_gb300 import synth

        def pinned(x):
            return torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()

        # the instances' CSR arrays in pinned host memory (copied before the timed region)
        inst_h = [(synth.Csr(pinned(d.row_ptr), pinned(d.col_idx), pinned(d.values), d.n_terms), k_, ids_)
                  for d, k_, ids_ in inst]
        t0 = time.perf_counter()
        for _ in range(args.steps):
            skm.fit_batched(inst_h, W.max_iter, tau=args.tau, use_graph=True, tune_cache=cache, device=local)
        e_dt = max_over_ranks(dist, time.perf_counter() - t0, dev)
        e2e = {"value": docs_done / e_dt, "unit": UNIT,
               "h2d_bytes_per_step": int(sum(8 * (d.n_docs + 1) + 8 * d.nnz for d, _, _ in inst)),
               "d2h_bytes_per_step": int(4 * n_total + 8 * W.max_iter * len(inst)), "host_memory": "pinned"}
    pk = peaks(device_sm_count(local))
    ach = 2.0 * fmas / (loop_ms / 1e3) / 1e12 if loop_ms > 0 else None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        docs0, k0, ids0 = max(inst, key=lambda x: x[0].nnz * x[1])
        C0 = np.zeros((docs0.n_terms, k0), np.float32)
        for j, i in enumerate(ids0):
            a, b = docs0.row_ptr[i], docs0.row_ptr[i + 1]
            C0[docs0.col_idx[a:b], j] = docs0.values[a:b]
        rate, n, cdt, cores = oracle_sample_rate(docs0, C0, 4243, args.cpu_budget)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} documents of the largest instance (k={k0}), one assignment step against its "
                         f"initial centroids, {cdt:.1f} s"}
    if os.path.exists(cache):
        os.remove(cache)
    if rank == 0:
        line = {"metric": METRIC, "value": docs_done / t_max, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(W.describe(), step="one skm_fit_batched call over all instances (setup + loop)",
                               docs_total=n_total, parallelism=f"replicas x{world}",
                               l2="inputs larger than L2", graph_nodes=st["graph_nodes"] if st else None,
                               shapes=st["shape_instances"] if st else None),
                "roofline": {"bound": "alu", "achieved": ach, "peak": pk["fp32_tflops"], "unit": "TFLOP/s",
                             "frac": ach / pk["fp32_tflops"] if ach else None, "traffic": None,
                             "peak_source": pk["fp32_source"],
                             "kernel": "whole iteration loop (all kernels; a lower bound for the scoring kernel)",
                             "loop_ms_per_step": loop_ms / args.steps},
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": None}
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving form
def sustained_rate(sweep, max_waiting: float = 0.1):
    """The largest offered rate of a sweep at which every assignment was served and at most
    max_waiting of the clustering jobs were still waiting at the end of the window (None if
    no rate qualifies)."""
    ok = [o["rate"] for o in sweep
          if o["assign_done"] == o["assign_requests"] and (o["fit_deferred_fraction"] or 0.0) <= max_waiting]
    return max(ok) if ok else None


def serving_session(W, local: int, window: float, tau: float, rates=None, job_slots: int = 2) -> dict:
    """Serving form: open-loop Poisson arrivals against skm_server for a fixed window on a
    resident BF16 centroid set under the workload's device budget. Returns the latency,
    throughput and admission figures at the workload's offered rate; with `rates`, also one
    window per rate (a fresh server each, same resident centroids) and the largest rate the
    server sustained: every assignment served and at most 10% of clustering jobs left waiting
    at the end of the window."""
    import torch

    from paper_2108_00895_gb300 import skm, synth
    dev = torch.device("cuda", local)
    pool = W.pool()
    # resident centroids: two Lloyd steps on the pool, loaded into an assignment-only context
    with skm.SphericalKMeans(W.k, precision="bf16", prune="ncc", max_iter=2, allocator="cuda", device=local) as tmp:
        tmp.fit(pool, synth.init_ids(pool.n_docs, W.k, 2000 + W.seed))
        C = tmp.centroids()
    stream = torch.cuda.Stream(dev)
    resident = skm.SphericalKMeans(W.k, precision="bf16", rescore=True, tau=tau, allocator="cuda",
                                   stream=stream.cuda_stream, device=local)
    resident.set_centroids(C)
    del C
    try:
        out = _serving_window(W, local, window, tau, resident, pool, W.rate, True, job_slots)
        if rates:
            sweep = []
            for r in rates:
                o = _serving_window(W, local, window, tau, resident, pool, float(r), False, job_slots)
                o.pop("queue_depth")
                o.pop("clocks")
                sweep.append(dict(rate=float(r), **o))
            out["rate_sweep"] = sweep
            out["sustained_rate"] = sustained_rate(sweep)
    finally:
        resident.close()
    return out


def _serving_window(W, local, window, tau, resident, pool, rate, sample_clocks, job_slots) -> dict:
    """One open-loop window at `rate` requests/s on a fresh server over `resident`."""
    import math

    from paper_2108_00895_gb300 import skm, synth
    budget = int(W.budget_gb * (1 << 30))
    srv = skm.Server(resident, budget, n_job_slots=job_slots, max_batch_docs=65536, max_batch_nnz=65536 * 300,
                     job_precision="bf16", job_prune="ncc", tau=tau, device=local)
    rng = np.random.default_rng(W.seed)
    rp, col, val = pool.row_ptr, pool.col_idx, pool.values

    def assign_req(n):
        a = int(rng.integers(0, pool.n_docs - n))
        return synth.Csr(rp[a:a + n + 1] - rp[a], col[rp[a]:rp[a + n]], val[rp[a]:rp[a + n]], pool.n_terms)

    def job_req():
        n = int(round(math.exp(rng.uniform(math.log(W.job_n_lo), math.log(W.job_n_hi)))))
        k = int(round(math.exp(rng.uniform(math.log(W.job_k_lo), math.log(W.job_k_hi)))))
        docs = synth.Csr(rp[:n + 1], col[:rp[n]], val[:rp[n]], pool.n_terms)   # prefix: zero copy
        ids = np.unique(np.linspace(0, n - 1, k).astype(np.int32))
        return docs, len(ids), ids

    # warm-up: a few requests of each kind
    for t in [srv.submit_assign(assign_req(64)) for _ in range(8)]:
        srv.wait(t)
    srv.wait(srv.submit_fit(synth.Csr(rp[:10001], col[:rp[10000]], val[:rp[10000]], pool.n_terms), 64,
                            np.arange(64, dtype=np.int32), 2))
    clocks = ClockSampler(local) if sample_clocks else None
    if clocks:
        clocks.start()
    tickets = []
    depth = []          # (seconds since start, assignments queued, jobs queued, jobs running)
    t0 = time.perf_counter()
    t_next = 0.0
    last_probe = -1.0
    while True:
        t_next += rng.exponential(1.0 / rate)
        if t_next > window:
            break
        now = time.perf_counter() - t0
        if t_next > now:
            time.sleep(t_next - now)
        if rng.random() < W.p_assign:
            n = int(round(math.exp(rng.uniform(0.0, math.log(W.assign_hi)))))
            tickets.append(("assign", n, srv.submit_assign(assign_req(n))))
        else:
            docs, k, ids = job_req()
            tickets.append(("fit", docs.n_docs, srv.submit_fit(docs, k, ids, W.job_iters)))
        if now - last_probe >= 0.5:
            st_ = srv.stats()
            depth.append((round(now, 2), int(st_["assign_queued"]), int(st_["fit_queued"]),
                          int(st_["jobs_running"])))
            last_probe = now
    t_submit_end = time.perf_counter() - t0
    lat_a, lat_f, docs_a, done_f, cl_docs, deferred, rejected = [], [], 0, 0, 0, 0, 0
    for kind, n, t in tickets:   # assignments drain within a short grace period
        if kind != "assign":
            continue
        res = srv.wait(t, timeout_ms=5000)
        if res is not None and res["state"] == "done":
            lat_a.append(res["latency_ms"])
            docs_a += n
    t_drain = time.perf_counter() - t0
    stats = srv.stats()
    for kind, n, t in tickets:
        if kind != "fit":
            continue
        res = srv.wait(t, timeout_ms=0)
        if res is None:
            deferred += 1
        elif res["state"] == "done":
            done_f += 1
            lat_f.append(res["latency_ms"])
            cl_docs += n * res["iters"]
        elif res["state"] == "rejected":
            rejected += 1
    clk = clocks.stop() if clocks else None
    srv.close()
    pct = lambda v, q: float(np.percentile(v, q)) if len(v) else None
    n_assign = sum(1 for k_, _, _ in tickets if k_ == "assign")
    n_fit = len(tickets) - n_assign
    return {"window_s": window, "assign_requests": n_assign, "assign_done": len(lat_a),
            "assign_p50_ms": pct(lat_a, 50), "assign_p99_ms": pct(lat_a, 99),
            "assign_docs_per_s": docs_a / t_drain,
            "offered_rate": rate, "offered_assign_docs_per_s": sum(n for k_, n, _ in tickets if k_ == "assign") / window,
            "fit_requests": n_fit, "fit_done": done_f, "fit_deferred_at_end": deferred,
            "fit_deferred_fraction": deferred / n_fit if n_fit else None,
            "fit_rejected": rejected, "fit_rejected_fraction": rejected / n_fit if n_fit else None,
            "fit_p50_ms": pct(lat_f, 50), "fit_p99_ms": pct(lat_f, 99),
            "clustered_docs_per_s": cl_docs / t_drain, "assign_batches": stats["assign_batches"],
            "max_batch_docs": stats["max_batch_docs_seen"], "peak_jobs_running": stats["peak_jobs_running"],
            "queue_depth": depth, "budget_gb": W.budget_gb, "resident_gb": stats["resident_mem"] / 2 ** 30,
            "submit_seconds": t_submit_end, "drain_seconds": t_drain, "clocks": clk}


def run_serving(args, world, rank, local, dist):
    """Serving form on its own: a window of args.serve_seconds."""
    import torch

    from paper_2108_00895_gb300 import skm, workloads
    W = workloads.SERVING
    torch.cuda.set_device(torch.device("cuda", local))
    skm.load()
    rates = [float(r) for r in args.serve_rates.split(",")] if args.serve_rates else None
    sv = serving_session(W, local, args.serve_seconds, args.tau, rates, args.serve_job_slots)
    clk = sv.pop("clocks")
    line = {"metric": "serving docs assigned/s; p50/p99 assignment latency (ms)", "value": sv["assign_docs_per_s"],
            "unit": "docs/s", "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * sv["drain_seconds"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": dict(W.describe(), window_s=args.serve_seconds, job_slots=args.serve_job_slots,
                           max_batch_docs=65536),
            "serving": sv, "clocks": clk,
            "e2e": {"value": sv["assign_docs_per_s"], "unit": "docs/s", "h2d_bytes_per_step": None,
                    "d2h_bytes_per_step": None}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["large", "medium", "small", "tweets", "abstracts", "batched", "serving"],
                    default="large")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="serving window (open loop)")
    ap.add_argument("--serve-rates", default="50,100,250,500,1000,2000,4000",
                    help="serving workload: also one window per offered rate (requests/s, comma list; '' = none)")
    ap.add_argument("--serve-job-slots", type=int, default=2, help="serving: clustering jobs run at once")
    ap.add_argument("--tau", type=float, default=1e-4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-checks", action="store_true",
                    help="skip the untimed checks (error against the oracle, FP32 full path, serving window)")
    ap.add_argument("--serve-check-seconds", type=float, default=3.0,
                    help="serving window of the default run's serving check (0 = none)")
    ap.add_argument("--profile-run", action="store_true",
                    help="allow fewer warm-up steps (launch lists under a profiler; not a timed number)")
    ap.add_argument("--precision", choices=["bf16", "fp32"], default=None, help="override the workload's")
    ap.add_argument("--prune", choices=["ncc", "none", "ncc_index"], default=None, help="override the workload's")
    ap.add_argument("--index-min-changed", type=int, default=100,
                    help="ncc_index: steps use the threshold index after more than this many centroids changed")
    ap.add_argument("--index-max-cands", type=int, default=256,
                    help="ncc_index: candidate cap of the index (documents with more are scored densely); "
                         "0 = the library's default, which runs the NCC passes alone")
    ap.add_argument("--rescore", choices=["on", "off"], default="on", help="FP64 rescoring of near ties")
    ap.add_argument("--max-iter", type=int, default=None, help="override the workload's step limit")
    ap.add_argument("--sparse-div", type=int, default=0, help="sparse centroid rows (0 = off)")
    ap.add_argument("--head-terms", type=int, default=0,
                    help="BF16: head terms scored on the tensor cores (0 = automatic, -1 = off)")
    ap.add_argument("--case", default=None, help="N,D,K: the workload's recipe at other sizes")
    ap.add_argument("--k", type=int, default=None, help="override the workload's number of clusters")
    args = ap.parse_args()
    if args.warmup < 3 and not args.profile_run:
        ap.error("--warmup must be >= 3 (timed numbers need three warm-up steps)")
    from paper_2108_00895_gb300 import workloads
    world, rank, local, dist = dist_setup(args)
    if args.workload == "serving":
        try:
            if args.impl == "reference":
                print(json.dumps({"impl": "reference", "unavailable": "the serving form has no CPU counterpart; "
                                  "the oracle arm is timed on the large workload"}))
            else:
                run_serving(args, world, rank, local, dist)
        finally:
            if dist is not None:
                dist.destroy_process_group()
        return
    if args.workload == "batched":
        try:
            if args.impl == "reference":
                if rank == 0:
                    W = workloads.BATCHED
                    inst = W.instances()
                    docs0, k0, ids0 = max(inst, key=lambda x: x[0].nnz * x[1])
                    C0 = np.zeros((docs0.n_terms, k0), np.float32)
                    for j, i in enumerate(ids0):
                        a, b = docs0.row_ptr[i], docs0.row_ptr[i + 1]
                        C0[docs0.col_idx[a:b], j] = docs0.values[a:b]
                    times = []
                    for s_ in range(args.warmup + args.steps):
                        rate, n, cdt, cores = oracle_sample_rate(docs0, C0, 100 + s_, 150.0 / (args.warmup + args.steps))
                        if s_ >= args.warmup:
                            times.append(rate)
                    value = float(np.mean(times))
                    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
                                      "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                                      "dtype": "f64", "data": "synthetic", "config": W.describe(),
                                      "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                                       "sample": f"{n} documents of the largest instance per step"},
                                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                              "d2h_bytes_per_step": 0}}), flush=True)
            else:
                run_batched(args, world, rank, local, dist)
        finally:
            if dist is not None:
                dist.destroy_process_group()
        return
    w = workloads.ALL[args.workload]
    over = {}
    if args.precision:
        over["precision"] = args.precision
    if args.prune:
        over["prune"] = args.prune
    if args.max_iter:
        over["max_iter"] = args.max_iter
    if args.case:
        n, d, k = (int(x) for x in args.case.split(","))
        over.update(n_docs=n, n_terms=d, k=k, name=f"{w.name} scaled to N={n} d={d} k={k}")
    if args.k:
        over.update(k=args.k, name=f"{over.get('name', w.name)} with k={args.k}")
    if over:
        w = w.scaled(**over)
    try:
        if args.impl == "reference":
            run_reference(args, w, world, rank, dist)
        else:
            run_ours(args, w, world, rank, local, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
