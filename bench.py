"""Benchmark: seconds per Lloyd iteration of inverted-file spherical k-means.

Default workload: 1,000,000 synthetic Zipf documents over 500,000 terms
(lognormal lengths, mean 120), K = 10,000, FP32 storage.  One step = one full
Lloyd iteration (assignment step + update step) through the C ABI; inputs are
resident in HBM when the timed region starts and are larger than L2 (CSR
0.96 GB).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--storage f32|f16|bf16]

--impl reference times the FP64 CPU oracle on the host cores instead (a
bounded sample of each iteration, scaled to the whole workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "sec/Lloyd iteration & assign-step HBM GB/s (% peak); mixed vs FP32 at equal assigns"
UNIT = "s/iter"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "assign_kernel_dram_traffic.txt")
# the assignment kernel's sources: counters taken on another version do not apply
ASSIGN_SRCS = [os.path.join(ROOT, "paper_2002_09094_gb300", "csrc", f) for f in ("assign.cu", "assign_common.cuh")]
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="ivf-scale-n1m-d500k-k10k")
    p.add_argument("--storage", choices=["f32", "f16", "bf16"], default="f32")
    p.add_argument("--n-docs", type=int, default=0, help="use only this many documents of the workload "
                   "(same generator; for small profiling cases)")
    p.add_argument("--k", type=int, default=0, help="override the number of clusters (profiling cases)")
    p.add_argument("--kernel", choices=["auto", "dense_head", "sparse", "tensor_head", "ivfd"], default="auto",
                   help="assignment kernel family (auto = the autotuner picks; ivfd = the comparison "
                        "algorithm IVFD, Algorithm 4)")
    p.add_argument("--instances", type=int, default=256, help="instances of --workload batched")
    p.add_argument("--e2e-steps", type=int, default=0,
                   help="steps of the end-to-end leg (0 = as many as --steps)")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle timing sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--schedule", choices=["auto", "tile_major", "object_major"], default="auto",
                   help="assignment schedule (auto = the autotuner picks)")
    p.add_argument("--no-mixed", action="store_true", help="skip the FP16/BF16 arms of the FP32 line")
    p.add_argument("--no-batched", action="store_true", help="skip the batched sub-line")
    p.add_argument("--batched-instances", type=int, default=32,
                   help="instances of the batched sub-line of the default line (0 = none)")
    p.add_argument("--batched-steps", type=int, default=8, help="timed iterations of the batched sub-line")
    p.add_argument("--fp64-sample", type=int, default=2000, help="objects checked against the FP64 oracle")
    return p.parse_args()


def e2e_steps(args) -> int:
    return args.e2e_steps if args.e2e_steps > 0 else max(1, args.steps)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def assign_sources_sha() -> str:
    """sha256 over the assignment kernel's source files, in order."""
    h = hashlib.sha256()
    for p in ASSIGN_SRCS:
        h.update(open(p, "rb").read())
    return h.hexdigest()


def traffic_per_launch(workload_name: str, storage: str, schedule: str | None = None, what: str = "bytes"):
    """DRAM bytes (what="bytes") or L2 bytes (what="l2_bytes") per assignment
    step from the committed ncu summary, or None when the kernel source
    changed since the counters were taken, the counters are for another
    workload, or they were taken under another schedule (tile-major or
    object-major) than the one in use."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    sha = assign_sources_sha()
    m_sha = re.search(r"assign_src_sha256:\s*([0-9a-f]+)", text)
    if not m_sha or m_sha.group(1) != sha:
        return None
    m_w = re.search(r"^workload:\s*(\S+)", text, re.M)
    if not m_w or m_w.group(1) != workload_name:
        return None
    m_s = re.search(rf"^schedule\[{storage}\]:\s*(\S+)", text, re.M)
    if m_s and schedule is not None and m_s.group(1) != schedule:
        return None
    m = re.search(rf"^{what}_per_launch\[{storage}\]:\s*([0-9.eE+]+)", text, re.M)
    return float(m.group(1)) if m else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t_begin: float, t_end: float):
        """Stop sampling; summarise the samples taken between t_begin and t_end
        (host wall clock).  The sampler starts before the warm-up, so its own
        start-up never overlaps the timed region."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [ln for ts, ln in self.lines if t_begin <= ts <= t_end + 0.25]
        for ln in inside:
            parts = [p.strip() for p in ln.split(",")]
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
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_iteration_sample(corpus, means, assign_for_update, rng, budget_s: float):
    """Time the FP64 oracle on a bounded sample and scale to the whole workload.

    Assignment: similarities + argmax for S sampled objects, scaled by N/S.
    Update: member sums + normalisation over the objects of a contiguous row
    range, scaled by nnz / nnz(range).  Returns (seconds per iteration, sample text).
    """
    import oracle.spherical_kmeans as sk
    from paper_2002_09094_gb300 import datagen as dg

    n = corpus.n_docs
    # size the sample from a short probe
    probe = rng.choice(n, size=min(n, 64), replace=False)
    t = time.perf_counter()
    sk.assign_from_similarities(sk.similarities(corpus, means, probe))
    per_obj = max((time.perf_counter() - t) / len(probe), 1e-7)
    s = int(min(n, max(64, 0.6 * budget_s / per_obj)))
    rows = rng.choice(n, size=s, replace=False)
    t = time.perf_counter()
    sk.assign_from_similarities(sk.similarities(corpus, means, rows))
    t_assign = (time.perf_counter() - t) * n / s
    # update over a leading row range: probe 1% of the rows, then grow the
    # range to about 40% of the budget
    def timed_update(hi):
        sub = dg.Corpus(row_ptr=corpus.row_ptr[:hi + 1].copy(), term=corpus.term[:corpus.row_ptr[hi]],
                        val=corpus.val[:corpus.row_ptr[hi]], n_terms=corpus.n_terms)
        t = time.perf_counter()
        sk.update(sub, assign_for_update[:hi], means)
        return time.perf_counter() - t, sub

    hi = max(1, n // 100)
    dt, sub = timed_update(hi)
    grow = 0.4 * budget_s / max(dt, 1e-4)
    if grow > 2.0 and hi < n:
        hi = int(min(n, hi * grow))
        dt, sub = timed_update(hi)
    t_update = dt * corpus.nnz / max(1, sub.nnz)
    desc = (f"oracle assignment of {s} random objects scaled x{n / s:.1f}; oracle update over the first "
            f"{hi} objects ({sub.nnz} tuples) scaled x{corpus.nnz / max(1, sub.nnz):.1f}")
    return t_assign + t_update, desc


def paper_method_iteration_sample(corpus, means, assign_for_update, rng, budget_s: float, threads: int):
    """Time Algorithm 3 in C (FP64, -O3; OpenMP over objects and clusters)
    on the host cores: the assignment on a sample of objects scaled to all
    of them, the update over all objects and clusters in full.
    Returns (seconds per iteration, threads used, sample text)."""
    import oracle.ivf_alg3 as calg3

    xi = calg3.InvertedFile.from_means(means)
    n = corpus.n_docs
    nt = threads if threads > 0 else calg3.threads_available()
    probe = rng.choice(n, size=min(n, 32 * nt), replace=False)
    t = time.perf_counter()
    calg3.assignment_step(corpus, xi, means.k, rows=probe, threads=nt)
    per_obj = max((time.perf_counter() - t) / len(probe), 1e-8)
    s = int(min(n, max(len(probe), 0.6 * budget_s / per_obj)))
    rows = rng.choice(n, size=s, replace=False)
    t = time.perf_counter()
    calg3.assignment_step(corpus, xi, means.k, rows=rows, threads=nt)
    t_assign = (time.perf_counter() - t) * n / s
    # update: the K x D dense passes dominate; above ~5e9 of them a leading
    # range of clusters is timed and scaled, over the cost of an empty range
    # (grouping objects by cluster and assembling the lists)
    k = means.k
    nc = int(min(k, max(16, 5e9 // max(1, corpus.n_terms))))
    t = time.perf_counter()
    calg3.update_step(corpus, assign_for_update, k, prev=xi, threads=nt, clusters=(0, nc))
    t_range = time.perf_counter() - t
    if nc < k:
        t = time.perf_counter()
        calg3.update_step(corpus, assign_for_update, k, prev=xi, threads=nt, clusters=(0, 0))
        t_fixed = time.perf_counter() - t
        t_update = t_fixed + max(0.0, t_range - t_fixed) * k / nc
        upd = f"update of {nc} of {k} clusters scaled x{k / nc:.1f} ({t_update:.2f} s)"
    else:
        t_update = t_range
        upd = f"update in full ({t_update:.2f} s)"
    desc = (f"Algorithm 3 in C on {nt} host thread(s): assignment of {s} random objects scaled x{n / s:.1f}, "
            + upd)
    return t_assign + t_update, nt, desc


def workload(args):
    from paper_2002_09094_gb300 import datagen as dg

    w = dg.WORKLOADS[args.workload]
    if args.n_docs or args.k:
        name = w.name + (f"-first{args.n_docs}" if args.n_docs else "") + (f"-k{args.k}" if args.k else "")
        w = w.scaled(n_docs=args.n_docs or None, k=args.k or None, name=name)
    return w


def max_over_ranks(value: float, dist, device: str) -> float:
    """Largest value over all ranks (the slowest replica sets the job time)."""
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def emit(obj):
    print(json.dumps(obj), flush=True)


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, on a bounded sample per step."""
    if rank != 0:
        return
    import oracle.spherical_kmeans as sk
    from paper_2002_09094_gb300 import datagen as dg

    w = workload(args)
    c = dg.make_corpus(w.corpus)
    ids = dg.init_doc_ids(c.n_docs, w.k, w.init_seed)
    means = sk.initial_means(c, ids)
    rng = np.random.default_rng(0)
    budget = max(2.0, min(args.cpu_seconds, 240.0 / max(1, args.steps + args.warmup)))
    assign_guess = rng.integers(0, w.k, size=c.n_docs).astype(np.int32)
    vals, desc = [], ""
    for step in range(args.warmup + args.steps):
        v, desc = oracle_iteration_sample(c, means, assign_guess, rng, budget)
        if step >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    cores = 1
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": {"workload": w.name, "n_docs": c.n_docs, "n_terms": c.n_terms, "nnz": c.nnz, "k": w.k,
                     "means": "seeded initial means (K documents), first iteration"},
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


def assign_roofline(c, w, storage, timing, info, l2_gbs, schedule):
    """Roofline of the assignment step (every launch of one step: one per
    cluster tile when tile-major, plus the pass over near-ties).

    achieved = algorithmic bytes (the CSR once, Eq. 15's posting entries at
    id + value bytes each, the outputs) / the step's kernel time.  Those
    bytes are served mostly by L2 (the hot lists stay resident), so the bound
    reported is L2, against the read bandwidth of a resident set measured live
    on this GPU (ivf_probe_l2_read).  Beside it: the DRAM bytes ncu counted
    for the same step (committed summary) as a fraction of the measured HBM
    peak, and the algorithmic bytes against HBM ("effective", above 1 when L2
    reuse is high)."""
    bv = 4 if storage == "f32" else 2
    n_steps = max(1, timing["n_assign"])
    kern_ms = timing["assign_kernel_ms"] / n_steps
    entries = timing["entries_visited"] / n_steps
    b_assign = c.nnz * (4 + bv) + 8 * (c.n_docs + 1) + entries * (2 + bv) + c.n_docs * 12
    hbm, hbm_kind = peaks()
    achieved = b_assign / (kern_ms / 1e3) / 1e9
    traffic = traffic_per_launch(w.name, storage, schedule)
    l2_bytes = traffic_per_launch(w.name, storage, schedule, what="l2_bytes")
    dram_gbs = traffic / (kern_ms / 1e3) / 1e9 if traffic else None
    return {"bound": "l2", "achieved": round(achieved, 1), "peak": round(l2_gbs, 1), "unit": "GB/s",
            "frac": round(achieved / l2_gbs, 4), "traffic": traffic,
            "peak_source": "L2 read bandwidth of a resident set, measured live on this GPU by ivf_probe_l2_read "
                           "(builder-measured; not a driver peak)",
            "kernel": ("assign step: k_build_xhead + k_tc_head (tcgen05) + k_assign" if info["dense_head_tensor"]
                       else "assign step: k_assign (%s)" % schedule),
            "algorithmic_bytes_per_launch": int(b_assign), "entries_per_launch": int(entries),
            "kernel_ms": round(kern_ms, 4),
            "l2_bytes_ncu": l2_bytes,
            "hbm": {"achieved": round(dram_gbs, 1) if dram_gbs else None, "peak": hbm, "unit": "GB/s",
                    "frac": round(dram_gbs / hbm, 4) if dram_gbs else None,
                    "peak_source": f"{hbm_kind} hbm_gbs (MEASURED_PEAKS.json)",
                    "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the step's launches"},
            "effective_vs_hbm": {"achieved": round(achieved, 1), "peak": hbm, "frac": round(achieved / hbm, 4),
                                 "label": "effective (L2 reuse): algorithmic bytes against HBM"}}


def mixed_arm(c, w, ids, storage, args, stream, cycles_total, a32_final):
    """FP16/BF16 storage on the same data and initial means: device-timed
    iterations, then as many assignments in all as the FP32 arm made, and its
    final assignment compared with the FP32 one object by object."""
    import torch

    from paper_2002_09094_gb300 import ivf

    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, w.k, storage=storage, stream=stream.cuda_stream) as m:
        m.set_means_from_docs(ids)
        for _ in range(args.warmup):
            m.assign(stats=False)
            m.update()
        torch.cuda.synchronize()
        m.timing_reset(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            m.assign(stats=False)
            m.update()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        timing = m.get_timing()
        m.timing_reset(False)
        info = m.info()
        done = args.warmup + args.steps
        st = None
        while done < cycles_total:
            st = m.assign()
            done += 1
            if done < cycles_total:
                m.update()
        a = m.get_assign()
        err = m.get_err_bound()
    n_steps = max(1, timing["n_assign"])
    return {"storage": storage, "value": ms / 1e3, "unit": UNIT, "ms_per_step": round(ms, 4),
            "phases_ms_per_step": {"assign_kernel": round(timing["assign_kernel_ms"] / n_steps, 4),
                                   "assign_step": round(timing["assign_step_ms"] / n_steps, 4),
                                   "update": round(timing["update_ms"] / max(1, timing["n_update"]), 4)},
            "rescored_per_step": round(timing["n_rescored"] / n_steps, 1),
            "kernel": kernel_desc(info),
            "assignments_vs_f32": {"assignments": cycles_total,
                                   "objects_differing": int(np.count_nonzero(a != a32_final)),
                                   "flagged_last": int(st["n_flagged"]) if st else None,
                                   "rescored_last": int(st["n_rescored"]) if st else None},
            "err_bound_last": {"max": float(err.max()), "median": float(np.median(err))}}


def kernel_desc(info):
    if not info["dense_head_r"]:
        return "sparse" + (" tile-major" if info.get("tile_major") else "")
    return "%s r=%d sub=%d theta=%.2f rows=%d%s" % (
        "tensor_head" if info["dense_head_tensor"] else "dense_head", info["dense_head_r"], info["dense_head_sub"],
        info["dense_head_theta"], info["dense_head_rows"], " tile-major" if info.get("tile_major") else "")


def fp64_sample_check(c, means, gpu_assign, gpu_best, gpu_err, rows):
    """Oracle similarities on a row sample (the CPU-baseline leg's sample):
    objects whose assignment differs from the FP64 argmax (gap >= 1e-6), and
    the measured |best - rho_FP64| against the GPU's per-object bound."""
    import oracle.spherical_kmeans as sk

    rho = sk.similarities(c, means, rows)
    a, best, gap = sk.assign_from_similarities(rho)
    ga = gpu_assign[rows]
    rho_g = rho[np.arange(len(rows)), ga]
    err = np.abs(gpu_best[rows].astype(np.float64) - rho_g)
    bound = gpu_err[rows].astype(np.float64)
    clear = gap >= 1e-6
    return {"objects": int(len(rows)), "assign_equal_fp64": int(np.count_nonzero((ga == a) & clear)),
            "excluded_near_ties": int(np.count_nonzero(~clear)),
            "differing": int(np.count_nonzero((ga != a) & clear)),
            "max_abs_err": float(err.max()), "max_err_over_bound": float((err / np.maximum(bound, 1e-30)).max()),
            "all_within_bound": bool(np.all(err <= bound + 1e-12))}


def run_ours(args, rank, world, local):
    import torch

    from paper_2002_09094_gb300 import build as cuda_build
    from paper_2002_09094_gb300 import datagen as dg
    from paper_2002_09094_gb300 import ivf

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    cuda_build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    w = workload(args)
    t0 = time.time()
    c = dg.make_corpus(w.corpus)
    gen_s = time.time() - t0
    ids = dg.init_doc_ids(c.n_docs, w.k, w.init_seed)
    stream = torch.cuda.Stream()
    bv = 4 if args.storage == "f32" else 2
    l2_gbs = ivf.probe_l2_read_gbs(stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        m = ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, w.k, storage=args.storage, stream=stream.cuda_stream,
                    kernel=args.kernel, schedule=args.schedule)
        m.set_means_from_docs(ids)
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        for _ in range(args.warmup):
            m.assign(stats=False)
            m.update()
        torch.cuda.synchronize()
        barrier()
        # ---------------------------------------------------------- timed region
        m.timing_reset(True)
        launches0 = ivf.launch_count()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier()
        t_begin = time.time()
        torch.cuda.nvtx.range_push("timed")  # lets ncu --nvtx-include "timed/" pick the timed launches
        step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev0.record(stream)
        step_ev[0].record(stream)
        for s_i in range(args.steps):
            m.assign(stats=False)
            m.update()
            step_ev[s_i + 1].record(stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        step_ms = [step_ev[q].elapsed_time(step_ev[q + 1]) for q in range(args.steps)]
        barrier()
        t_end = time.time()
        total_ms = ev0.elapsed_time(ev1)
        launches = ivf.launch_count() - launches0
        clk = clocks.stop(t_begin, t_end)
        timing = m.get_timing()
        m.timing_reset(False)
        info = m.info()
        if dist is not None:
            total_ms = max_over_ranks(total_ms, dist, "cuda")
        # ------------------------------------------------------ end to end
        # each step: host->device copy of the objects from pinned memory, one
        # iteration, device->host read of the assignment.  The copy of step
        # i + 1 is issued once step i's assignment is enqueued, so it runs on
        # the context's copy stream while that assignment computes; the first
        # step's copy is not overlapped.
        rp_h = torch.from_numpy(c.row_ptr).pin_memory()
        tm_h = torch.from_numpy(c.term).pin_memory()
        vl_h = torch.from_numpy(c.val).pin_memory()
        out_h = torch.empty(c.n_docs, dtype=torch.int32).pin_memory()
        h2d = rp_h.numel() * 8 + tm_h.numel() * 4 + vl_h.numel() * 4
        d2h = out_h.numel() * 4
        # one untimed step first (the context allocates its staging copy of
        # the objects on the first load)
        m.load_objects(rp_h, tm_h, vl_h)
        m.assign(stats=False)
        m.update()
        m.get_assign(out_h)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m.load_objects(rp_h, tm_h, vl_h)
        n_e2e = e2e_steps(args)
        for q in range(n_e2e):
            m.assign(stats=False)
            if q + 1 < n_e2e:
                m.load_objects(rp_h, tm_h, vl_h)
            m.update()
            m.get_assign(out_h)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1) / n_e2e
        cycles_total = args.warmup + args.steps + 1 + n_e2e
        # the state of the last assignment: the means it used are the ones
        # before its update, so the FP64 check below re-runs that assignment
        means_np = m.get_means()
        st_last = m.assign()
        assign_np, best_np, err_np = m.get_assign(), m.get_best(), m.get_err_bound()
        m.close()
        mixed = []
        if args.storage == "f32" and not args.no_mixed:
            for st in ("bf16", "f16"):
                mixed.append(mixed_arm(c, w, ids, st, args, stream, cycles_total + 1, assign_np))
        batched = None
        if not args.no_batched and args.batched_instances > 0:
            batched = measure_batched(args, args.batched_instances, stream)

    ms_per_step = total_ms / args.steps
    n_steps = max(1, timing["n_assign"])
    schedule = "tile_major" if info.get("tile_major") else "object_major"
    roof = assign_roofline(c, w, args.storage, timing, info, l2_gbs, schedule)
    out = {"metric": METRIC, "value": ms_per_step / 1e3 / world, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
           "data": "synthetic", "impl": "ours",
           "config": {"workload": w.name, "n_docs": c.n_docs, "n_terms": c.n_terms, "nnz": c.nnz, "k": w.k,
                      "storage": args.storage, "parallelism": "replicas" if world > 1 else "single",
                      "l2": "inputs larger than L2 (CSR %.2f GB); no flush" % (c.nnz * 8 / 1e9),
                      "k_tile": info["k_tile"], "warps_per_block": info["warps_per_block"],
                      "kernel": kernel_desc(info), "schedule": schedule,
                      "ivf_entries": info["ivf_entries"], "generation_s": round(gen_s, 1)},
           "step_ms": {"min": round(min(step_ms), 3), "median": round(statistics.median(step_ms), 3),
                       "max": round(max(step_ms), 3)},
           "phases_ms_per_step": {"assign_kernel": round(timing["assign_kernel_ms"] / n_steps, 4),
                                  "assign_step": round(timing["assign_step_ms"] / n_steps, 4),
                                  "update": round(timing["update_ms"] / max(1, timing["n_update"]), 4)},
           "rescored_per_step": round(timing["n_rescored"] / n_steps, 1),
           "roofline": roof,
           "e2e": {"value": e2e_ms / 1e3 / world, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(d2h), "steps": n_e2e},
           "gpu_launches": int(launches), "clocks": clk,
           "err_bound_last": {"max": float(err_np.max()), "median": float(np.median(err_np)),
                              "flagged": int(st_last["n_flagged"]), "rescored": int(st_last["n_rescored"])}}
    if mixed:
        out["mixed_precision"] = {
            "note": "same data and initial means; value = device-timed s/iter; assignments compared with the "
                    "FP32 arm after the same number of assignments",
            **{a["storage"]: {**a, "speedup_vs_f32": round(ms_per_step / a["ms_per_step"], 3)} for a in mixed}}
    if batched is not None:
        out["batched"] = batched
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle.spherical_kmeans as sk

        ptr, term, val = means_np
        means = sk.Means(ptr=ptr, term=term.astype(np.int64), val=val, n_terms=c.n_terms)
        v, desc = oracle_iteration_sample(c, means, assign_np, np.random.default_rng(1), args.cpu_seconds)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": desc + "; means = the GPU's current FP64 means"}
        # the last assignment against the FP64 argmax on a sample, and the
        # measured error of each best against the GPU's own per-object bound
        rows = np.random.default_rng(3).choice(c.n_docs, size=min(c.n_docs, args.fp64_sample), replace=False)
        out["fp64_check"] = fp64_sample_check(c, means, assign_np, best_np, err_np, np.sort(rows))
        # the paper's own method on the same host, one thread (as the paper
        # runs it) and every core
        pm = {}
        for label, nt in (("one_thread", 1), ("all_threads", 0)):
            v, used, desc = paper_method_iteration_sample(c, means, assign_np, np.random.default_rng(2),
                                                          args.cpu_seconds / 2, nt)
            pm[label] = {"value": v, "unit": UNIT, "cores": used, "sample": desc}
        out["cpu_paper_method"] = {"kind": "Algorithm 3 (IVF) in C, FP64, gcc -O3", **pm}
    if rank == 0:
        emit(out)
    if dist is not None:
        dist.destroy_process_group()


def measure_batched(args, n_instances, stream):
    """Many independent instances of uneven N, K and D in one context (one
    launch per phase for all of them, CUDA-graph iterations) against the same
    instances run one after the other in their own contexts.  Returns the
    batched line's fields."""
    import torch

    from paper_2002_09094_gb300 import datagen as dg
    from paper_2002_09094_gb300 import ivf

    ws = dg.batched_workloads(n_instances=n_instances)
    t0 = time.time()
    cs = [dg.make_corpus(w.corpus) for w in ws]
    gen_s = time.time() - t0
    ids = [dg.init_doc_ids(c.n_docs, w.k, w.init_seed) for w, c in zip(ws, cs)]
    inst_docs = np.concatenate([[0], np.cumsum([c.n_docs for c in cs])]).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum([c.nnz for c in cs])]).astype(np.int64)
    row_ptr = np.concatenate([c.row_ptr[:-1] + o for c, o in zip(cs, offs)] + [offs[-1:]]).astype(np.int64)
    term = np.concatenate([c.term for c in cs])
    val = np.concatenate([c.val for c in cs])
    iters = args.batched_steps
    storage = "f32"
    with torch.cuda.stream(stream):
        m = ivf.BatchedIVF(row_ptr, term, val, inst_docs, [c.n_terms for c in cs], [w.k for w in ws],
                           storage=storage, stream=stream.cuda_stream)
        del term, val
        m.set_means_from_docs(np.concatenate(ids))
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        m.iterate(args.warmup)
        launches0 = ivf.launch_count()
        torch.cuda.synchronize()
        t_begin = time.time()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        done, conv, st = m.iterate(iters)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop(t_begin, time.time())
        batched_ms = e0.elapsed_time(e1) / max(1, done)
        launches = ivf.launch_count() - launches0
        a_batched = m.get_assign()
        info = m.info()
        # phase split from one more (eager, event-timed) iteration, outside the timed region
        m.timing_reset(True)
        m.assign(stats=False)
        m.update()
        torch.cuda.synchronize()
        tph = m.get_timing()
        m.timing_reset(False)
        m.close()
        # the same instances, one context each, same iterations
        seq_ms = 0.0
        seq_ph = {"assign_kernel": 0.0, "assign_step": 0.0, "update": 0.0}
        equal = True
        for b, (w, c, d) in enumerate(zip(ws, cs, ids)):
            with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, w.k, storage=storage,
                         stream=stream.cuda_stream) as s1:
                s1.set_means_from_docs(d)
                s1.iterate(args.warmup)
                torch.cuda.synchronize()
                f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                f0.record(stream)
                s1.iterate(done)
                f1.record(stream)
                torch.cuda.synchronize()
                seq_ms += f0.elapsed_time(f1) / max(1, done)
                equal &= bool(np.array_equal(s1.get_assign(), a_batched[inst_docs[b]:inst_docs[b + 1]]))
                s1.timing_reset(True)
                s1.assign(stats=False)
                s1.update()
                torch.cuda.synchronize()
                t1 = s1.get_timing()
                s1.timing_reset(False)
                for key in seq_ph:
                    seq_ph[key] += t1[key + "_ms"]
    n_all, nnz_all = int(inst_docs[-1]), int(offs[-1])
    return {"workload": f"batched-{n_instances}-instances", "instances": n_instances, "n_docs": n_all,
            "nnz": nnz_all, "k_total": int(sum(w.k for w in ws)), "storage": storage,
            "value": batched_ms / 1e3, "unit": UNIT, "ms_per_step": round(batched_ms, 4), "steps": int(done),
            "iterations": "graph-captured", "generation_s": round(gen_s, 1),
            "phases_ms_one_eager_iteration": {"assign_kernel": round(tph["assign_kernel_ms"], 3),
                                              "assign_step": round(tph["assign_step_ms"], 3),
                                              "update": round(tph["update_ms"], 3)},
            "kernel": kernel_desc(info),
            "sequential_s_per_iter": seq_ms / 1e3, "batched_speedup": round(seq_ms / batched_ms, 3),
            "sequential_phases_ms_one_eager_iteration": {k_: round(v_, 3) for k_, v_ in seq_ph.items()},
            "equal_assignments": equal, "converged": bool(conv), "gpu_launches": int(launches), "clocks": clk,
            "entries_one_eager_iteration": int(tph["entries_visited"])}


def run_batched(args, rank, world, local):
    """The batched workload as the line's own metric (--workload batched)."""
    import torch

    from paper_2002_09094_gb300 import build as cuda_build

    cuda_build.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    args.batched_steps = args.steps
    b = measure_batched(args, args.instances, stream)
    out = {"metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": world, "steps": b["steps"],
           "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "ours",
           "config": {k_: b[k_] for k_ in ("workload", "instances", "n_docs", "nnz", "k_total", "storage",
                                            "iterations", "generation_s", "kernel")},
           "batched": b, "e2e": None, "gpu_launches": b["gpu_launches"], "clocks": b["clocks"]}
    if rank == 0:
        emit(out)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched":
        run_batched(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
