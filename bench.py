"""Benchmark of the TREVR2 reverse ray trace on one GB300 (or N in replica).

One step = one radiation step of the whole path on the clumpy multi-band
field: tree build (Morton keys, sort, bisection, aggregates, per-direction
absorption tables) + the walk giving J for every active receiver, 3 bands,
192 HEALPix beams.  The metric is active-receiver x beam x band per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun), each rank runs an independent snapshot (seed + rank):
weak scaling, no collective on the data path; the step time is the max over
ranks.  `--impl reference` times the FP64 CPU oracle on a bounded sample.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "active receiver x HEALPix-ray x band / s"
UNIT = "receiver*ray*band/s"
NODE_BYTES = 32  # walk record of one node
# The ncu summary of the walk kernel on the 96^3 version of the benchmark
# field records its DRAM bytes per launch and a hash of the sources the
# kernel is compiled from; the bench scales the bytes by receivers, and only
# while the sources still hash the same.
WALK_PROFILE = os.path.join(ROOT, "profiles", "k_walk_clumpy96.md")
WALK_SOURCES = ["walk.cu", "walk.cuh", "healpix.cuh", "internal.cuh"]


def kernel_sources_sha256():
    """SHA-256 over the sources compiled into the walk kernel (and the ABI
    header they include)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2310_15235_gb300", "csrc")
    for name in WALK_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    with open(os.path.join(ROOT, "include", "trevr2.h"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()


def _walk_profile_record():
    """The walk profile's machine-readable record, or (None, why)."""
    import re
    try:
        with open(WALK_PROFILE) as f:
            m = re.search(r"<!-- traffic (\{.*?\}) -->", f.read())
        rec = json.loads(m.group(1))
    except Exception:
        return None, "no machine-readable traffic record in the walk profile"
    if rec.get("sources_sha256") != kernel_sources_sha256():
        return None, ("the walk profile was captured on other kernel sources "
                      f"(sha256 {rec.get('sources_sha256', '?')[:12]}); capture it again")
    return rec, None


def _walk_traffic(receivers):
    """(DRAM bytes of one walk launch over `receivers` scaled from the
    profile's capture, note); bytes is None when the profile is missing or
    was taken on other kernel sources."""
    rec, why = _walk_profile_record()
    if rec is None:
        return None, why
    per = (rec["dram_read_bytes"] + rec["dram_write_bytes"]) / rec["receivers"]
    return per * receivers, (f"ncu dram bytes of one k_walk launch on the {rec['field']} "
                             f"({rec['receivers']:,} receivers), scaled by receivers; "
                             f"profiles/k_walk_clumpy96.md")


def _walk_counters(hbm_peak):
    """What the walk's ncu capture measured (DRAM throughput against the
    peak, L2 hit rate, warp execution efficiency, issue-active share), or
    None."""
    rec, _ = _walk_profile_record()
    if rec is None or "duration_ms" not in rec:
        return None
    gbs = (rec["dram_read_bytes"] + rec["dram_write_bytes"]) / (rec["duration_ms"] * 1e-3) / 1e9
    return {"field": rec["field"], "dram_gbs": gbs, "dram_frac": gbs / hbm_peak,
            "l2_hit_pct": rec["l2_hit_pct"],
            "warp_execution_efficiency": rec["lanes_active"] / 32.0,
            "issue_active_pct": rec["issue_active_pct"],
            "note": "ncu counters of one cold, serialised launch; the walk is bound by "
                    "instruction issue, not by DRAM"}


def _workload_name(case):
    n_gas = len(case["active"])
    return (f"clumpy multi-band field: {n_gas:,} gas on a 128^3 jittered lattice (lognormal, "
            f"sigma 1.5, P(k)~k^-3) + 10,000 power-law sources, 3 bands kappa (10, 3, 0.5), "
            f"nside 4 (192 beams), theta 0.5, all gas active")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
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
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _algorithmic_bytes_per_receiver(stats, nb):
    """Bytes a receiver's walk must touch by the method's own count:
    N_visit node records, one absorption value per band per beam segment,
    one source record (position + per-band luminosity) per source, and the
    J row written."""
    visited, cut, segments, sources = [stats[:, i].astype(np.float64) for i in range(4)]
    per = visited * NODE_BYTES + segments * 4 * nb + sources * (12 + 4 * nb) + 4 * nb
    return float(per.mean()), {k: float(v.mean()) for k, v in
                               zip(("visited", "cut", "segments", "sources"),
                                   (visited, cut, segments, sources))}


def _oracle_sample(case, seconds_target, rng_seed=0):
    """The FP64 oracle on a bounded sample of receivers (all host cores)."""
    import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ot = oracle.OracleTree.from_case(case)
    ot.alpha_table(case["nside"])  # builds and caches the tables
    t_build = time.perf_counter() - t0
    rng = np.random.default_rng(rng_seed)
    pilot = rng.choice(case["active"], 256, replace=False)
    t0 = time.perf_counter()
    _, st_p = ot.J(pilot, case["nside"], case["theta"], nthreads=cores, stats=True)
    t_p = time.perf_counter() - t0
    n = int(min(len(case["active"]), max(256, seconds_target / max(t_p, 1e-6) * 256)))
    sample = rng.choice(case["active"], n, replace=False)
    t0 = time.perf_counter()
    _, st = ot.J(sample, case["nside"], case["theta"], nthreads=cores, stats=True)
    t_j = time.perf_counter() - t0
    return ot, sample, st, t_j, t_build, cores


def run_reference(args, world, rank):
    if rank != 0:
        return
    case = workloads.clumpy_multiband()
    npix, nb = 12 * case["nside"] ** 2, case["nb"]
    import oracle
    cores = os.cpu_count() or 1
    ot = oracle.OracleTree.from_case(case)
    ot.alpha_table(case["nside"])
    rng = np.random.default_rng(1)
    per_step = args.reference_sample
    times = []
    for step in range(args.warmup + args.steps):
        sample = rng.choice(case["active"], per_step, replace=False)
        t0 = time.perf_counter()
        ot.J(sample, case["nside"], case["theta"], nthreads=cores)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    t = float(np.mean(times))
    value = per_step * npix * nb / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": _workload_name(case), "receivers_per_step": per_step,
                   "beams": npix, "bands": nb},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} random receivers per step of the 2,097,152; "
                                   f"tree and tables built once before timing"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch

    import paper_2310_15235_gb300 as t2

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    case = workloads.clumpy_multiband(seed=1003 + rank)
    npix, nb = 12 * case["nside"] ** 2, case["nb"]
    A = len(case["active"])
    units = A * npix * nb

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    inp = {k: to_dev(case[k]) for k in ("pos", "mass", "kappa", "lum", "h", "active")}
    J = torch.empty((A, nb), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev_walk=None):
        tree = t2.build(inp["pos"], inp["mass"], inp["kappa"], inp["lum"], inp["h"],
                        case["box_lo"], case["box_size"], case["bucket"], device=dev)
        tree.prepare(case["nside"])  # per-direction tables: part of the step
        if ev_walk is not None:
            ev_walk[0].record(stream)
        tree.J(inp["active"], case["nside"], case["theta"], out=J, flags=t2.ASYNC)
        if ev_walk is not None:
            ev_walk[1].record(stream)
        tree.status()
        tree.free()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = t2.kernel_launches()
    walk_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(walk_events[k])
    e1.record(stream)
    torch.cuda.synchronize()
    launches = t2.kernel_launches() - launches0
    clk = clocks.stop()
    total_ms = e0.elapsed_time(e1)
    walk_ms = [a.elapsed_time(b) for a, b in walk_events]
    ms_step = total_ms / args.steps
    if dist:
        t = torch.tensor([ms_step], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = world * units / (ms_step * 1e-3)

    # End to end through the public API from pinned host buffers.
    host = {k: torch.from_numpy(np.ascontiguousarray(case[k])).pin_memory()
            for k in ("pos", "mass", "kappa", "lum", "h", "active")}
    J_host = torch.empty((A, nb), dtype=torch.float32).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = J_host.numel() * 4

    def e2e_step():
        d = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
        tree = t2.build(d["pos"], d["mass"], d["kappa"], d["lum"], d["h"], case["box_lo"],
                        case["box_size"], case["bucket"], device=dev)
        out = tree.J(d["active"], case["nside"], case["theta"])
        J_host.copy_(out, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        tree.free()

    e2e_step()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / args.steps
    if dist:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * units / e2e_s

    if rank != 0:
        dist.destroy_process_group()
        return

    hbm_peak, peak_kind = _peaks()
    walk_avg = float(np.mean(walk_ms))
    roofline = None
    cpu = None
    extra = {}
    if world == 1 and not args.no_cpu_baseline:
        ot, sample, st, t_j, t_build, cores = _oracle_sample(case, args.cpu_seconds)
        per_rec, means = _algorithmic_bytes_per_receiver(st, nb)
        achieved = per_rec * A / (walk_avg * 1e-3) / 1e9
        traffic, traffic_note = _walk_traffic(A)
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": traffic,
                    "traffic_note": traffic_note, "ncu": _walk_counters(hbm_peak),
                    "kernel": "k_walk", "peak_kind": peak_kind,
                    "algorithmic_bytes_per_unit": per_rec / (npix * nb),
                    "per_receiver_counts": means}
        t0 = time.perf_counter()
        ot.J(sample[:256], case["nside"], case["theta"], nthreads=1)
        t_one = time.perf_counter() - t0
        cpu = {"value": len(sample) * npix * nb / t_j, "unit": UNIT, "cores": cores,
               "kind": "oracle",
               "sample": f"{len(sample)} random receivers of the same field (J walk only; "
                         f"oracle tree+tables build {t_build:.1f} s not included)",
               "single_thread": {"value": 256 * npix * nb / t_one, "unit": UNIT,
                                 "sample": "256 of the same receivers on one thread"}}
        # sampled parity of this very run
        ref = ot.J(sample[:512], case["nside"], case["theta"], nthreads=cores)
        idx = sample[:512]  # active == arange for this workload
        got = J.cpu().numpy()[idx]
        rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
        extra["parity_sample"] = {"receivers": 512, "median_rel": float(np.median(rel)),
                                  "max_rel": float(rel.max())}
        if not args.no_bucket:
            extra["bucket"] = run_bucket(case, inp, dev, walk_avg)
            ref = ot.J(sample[:256], case["nside"], case["theta"], flags=t2.BUCKET,
                       nthreads=cores)
            got = extra["bucket"].pop("_J")[sample[:256]]
            rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
            extra["bucket"]["parity_sample"] = {"receivers": 256,
                                                "median_rel": float(np.median(rel)),
                                                "max_rel": float(rel.max())}
            # a receiver's per-bucket counts are its bucket's walk
            _, st_b = ot.J(sample[:256], case["nside"], case["theta"], flags=t2.BUCKET,
                           nthreads=cores, stats=True)
            per_walk, means_b = _algorithmic_bytes_per_receiver(st_b, nb)
            per_eval = float(st_b[:, 3].mean()) * 16 + 4 * nb
            extra["bucket"]["per_walk_counts"] = means_b
            extra["_bucket_bytes"] = (per_walk, per_eval)
            # the paper's full near field: p-p absorption inside r_pp, the
            # receiver's own column by Eq. taucorr
            pp_flags = t2.PP | t2.THICK
            extra["bucket_pp"] = run_bucket(case, inp, dev, walk_avg, reps=2,
                                            extra_flags=pp_flags, kernel="k_walk_bucket (p-p)")
            ref = ot.J(sample[:128], case["nside"], case["theta"],
                       flags=t2.BUCKET | pp_flags, nthreads=cores)
            got = extra["bucket_pp"].pop("_J")[sample[:128]]
            rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
            extra["bucket_pp"]["parity_sample"] = {"receivers": 128,
                                                   "median_rel": float(np.median(rel)),
                                                   "max_rel": float(rel.max())}
            # the complex source model (tables built in the warm-up call)
            extra["bucket_csm"] = run_bucket(case, inp, dev, walk_avg, reps=2,
                                             extra_flags=t2.CSM, kernel="k_walk_bucket (CSM)")
            ref = ot.J(sample[:128], case["nside"], case["theta"], flags=t2.BUCKET | t2.CSM,
                       nthreads=cores)
            got = extra["bucket_csm"].pop("_J")[sample[:128]]
            rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
            extra["bucket_csm"]["parity_sample"] = {"receivers": 128,
                                                    "median_rel": float(np.median(rel)),
                                                    "max_rel": float(rel.max())}
    elif world == 1 and not args.no_bucket:
        extra["bucket"] = run_bucket(case, inp, dev, walk_avg)
        extra["bucket"].pop("_J")
        extra["bucket_pp"] = run_bucket(case, inp, dev, walk_avg, reps=2,
                                        extra_flags=t2.PP | t2.THICK,
                                        kernel="k_walk_bucket (p-p)")
        extra["bucket_pp"].pop("_J")
        extra["bucket_csm"] = run_bucket(case, inp, dev, walk_avg, reps=2,
                                         extra_flags=t2.CSM, kernel="k_walk_bucket (CSM)")
        extra["bucket_csm"].pop("_J")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": _workload_name(case), "receivers": A, "beams": npix, "bands": nb,
                   "step": "tree build + per-direction tables + walk (J)",
                   "l2": "inputs larger than L2 (elements, tree and alpha tables > 129 MB, "
                         "rebuilt every step)",
                   "parallelism": f"replicas x{world}"},
        "walk_ms": walk_avg, "walk_units_per_s": world * units / (walk_avg * 1e-3),
        "build_ms": ms_step - walk_avg,
        "adjoint_forward_ratio": None,
        "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "paper_context": {
            "value": 1.104175e6 * 48 * 1 / 3.4, "unit": UNIT,
            "note": "derived from the paper's Sec. 3.1 timing: one TREVR2 radiation step of "
                    "the MUGS2 galaxy (1,104,175 gas, 48 rays, 1 band) in 3.4 s on 320 CPU "
                    "cores, its per-bucket rays counted per receiver; another machine, "
                    "workload and scheme, so context only"},
    }
    if world == 1 and not args.no_adjoint:
        line["adjoint"] = run_adjoint(args, dev)
        line["adjoint_forward_ratio"] = line["adjoint"]["ratio"]
        line["adjoint"]["clumpy_2M"] = run_adjoint_clumpy(case, inp, dev)
    if world == 1 and not args.no_batched:
        per_rec = roofline["algorithmic_bytes_per_unit"] * npix * nb if roofline else None
        per_bucket, per_eval = extra.pop("_bucket_bytes", (None, None))
        line["batched"] = run_batched(args, dev, per_rec, per_bucket, per_eval, hbm_peak,
                                      peak_kind)
    line.update(extra)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _leaf_lookup(tree):
    """Maps receivers to the leaf holding them (each leaf is a contiguous
    range of the tree's sorted elements)."""
    perm = tree.export("perm").cpu().numpy()
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm), dtype=perm.dtype)
    child = tree.export("child").cpu().numpy()
    first = tree.export("first").cpu().numpy()
    count = tree.export("count").cpu().numpy()
    firsts = np.sort(first[(child < 0) & (count > 0)])
    return lambda receivers: np.searchsorted(firsts, inv[receivers], side="right") - 1


def _distinct_buckets(leaf_of, receivers):
    return int(len(np.unique(leaf_of(receivers))))


def _batched_arm(args, dev, trees, act, offsets, tree_of, members, outs, J, nside, theta, flags):
    """One plan (autotuned, recorded in a CUDA graph, replayed) against one
    plain trevr2_J launch per subset with the same flags on the same stream."""
    import torch

    import paper_2310_15235_gb300 as t2

    stream = torch.cuda.current_stream()
    plan = t2.Batch(trees, offsets, tree_of, nside=nside, theta=theta, flags=flags)
    warps, staging = plan.autotune(act, J)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.run(act, J)
    graph.replay()  # warm-up
    torch.cuda.synchronize()
    plan.status()
    reps = max(1, args.batched_reps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    plan.status()
    batched_ms = e0.elapsed_time(e1) / reps
    J_batched = J.clone()
    plan.free()
    del graph
    big = int(np.argmax(np.diff(offsets)))
    for t in range(len(trees)):  # walk buffers of every tree at their largest size
        s = max((s for s in range(len(members)) if tree_of[s] == t),
                key=lambda s: offsets[s + 1] - offsets[s])
        trees[t].J(members[s], nside, theta, out=outs[s], flags=t2.ASYNC | flags)
    trees[tree_of[big]].status()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        for s in range(len(members)):
            if len(members[s]):
                trees[tree_of[s]].J(members[s], nside, theta, out=outs[s],
                                    flags=t2.ASYNC | flags)
    e1.record(stream)
    torch.cuda.synchronize()
    for tr in trees:
        tr.status()
    plain_ms = e0.elapsed_time(e1) / reps
    # rows are trevr2_J's bit for bit at the plain path's staging depth (1024
    # sources per warp); another depth splits a receiver's sources into other
    # passes, so the sums may round differently
    same = bool(torch.equal(J, J_batched))
    rel = ((J_batched - J).abs() / J.abs().clamp_min(1e-30)).max().item()
    return {"batched_ms": batched_ms, "plain_ms": plain_ms, "speedup_vs_plain": plain_ms / batched_ms,
            "autotuned": {"warps_per_block": warps, "staged_sources_per_warp": staging},
            "rows_equal_to_plain": same, "rows_max_rel_vs_plain": rel, "reps": reps}


def run_batched(args, dev, per_receiver_bytes, per_bucket_walk_bytes, per_receiver_eval_bytes,
                hbm_peak, peak_kind):
    """Individual-timestep batching (Sec. 1.2, Sec. 3.1): 4 snapshots of the
    clumpy 2M field, 64 subsets each of 10^U(2,6) receivers.  The batch is one
    autotuned persistent launch replayed from a CUDA graph; the comparison is
    one plain trevr2_J launch per subset on the same stream with the same
    flags.  Measured per receiver (the walk of trevr2_J) and per bucket
    (TREVR2_BUCKET, the paper's own scheme, where a run walks each distinct
    (snapshot, bucket) once)."""
    import torch

    import paper_2310_15235_gb300 as t2

    snaps, subsets = workloads.batched_cases()
    nside, theta, nb = snaps[0]["nside"], snaps[0]["theta"], snaps[0]["nb"]
    npix = 12 * nside ** 2
    trees = []
    for c in snaps:
        d = {k: torch.from_numpy(np.ascontiguousarray(c[k])).to(dev)
             for k in ("pos", "mass", "kappa", "lum", "h")}
        tr = t2.build(d["pos"], d["mass"], d["kappa"], d["lum"], d["h"], c["box_lo"],
                      c["box_size"], c["bucket"], device=dev)
        tr.prepare(nside)
        trees.append(tr)
    offsets = np.zeros(len(subsets) + 1, np.int64)
    offsets[1:] = np.cumsum([len(m) for _, m in subsets])
    tree_of = np.array([t for t, _ in subsets], np.int32)
    act = torch.from_numpy(np.concatenate([m for _, m in subsets])).to(dev)
    total = int(offsets[-1])
    units = total * npix * nb
    J = torch.empty((total, nb), dtype=torch.float32, device=dev)
    members = [act[offsets[s]:offsets[s + 1]] for s in range(len(subsets))]
    outs = [J[offsets[s]:offsets[s + 1]] for s in range(len(subsets))]
    per_snap = [np.unique(np.concatenate([m for t, m in subsets if t == s]))
                for s in range(len(snaps))]
    distinct = sum(len(u) for u in per_snap)
    leaf_of = [_leaf_lookup(tr) for tr in trees]
    buckets = sum(_distinct_buckets(leaf_of[s], per_snap[s]) for s in range(len(snaps)))
    plain_bucket_walks = sum(_distinct_buckets(leaf_of[t], m) for t, m in subsets if len(m))

    rx = _batched_arm(args, dev, trees, act, offsets, tree_of, members, outs, J, nside, theta, 0)
    bk = _batched_arm(args, dev, trees, act, offsets, tree_of, members, outs, J, nside, theta,
                      t2.BUCKET)

    def roof(nbytes, ms, counts, note):
        if nbytes is None:
            return None
        achieved = nbytes / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_kind": peak_kind, "counts": counts,
                "note": note}

    out = {
        "workload": "4 clumpy 2,097,152-element 3-band snapshots (seeds 1040-1043), 64 subsets "
                    "each of floor(10^U(2,6)) receivers drawn without replacement, nside 4, "
                    "theta 0.5",
        "subsets": len(subsets), "receivers": total, "units": units,
        "distinct_receivers": int(distinct),
        "launch": "one CUDA graph: row keys, radix sort, distinct (tree, receiver) keys, one "
                  "persistent walk kernel over the distinct ones, scatter to rows",
        "plain_launches": int(sum(1 for m in members if len(m))),
        **rx,
        "batched_units_per_s": units / (rx["batched_ms"] * 1e-3),
        "plain_units_per_s": units / (rx["plain_ms"] * 1e-3),
        "roofline": roof(None if per_receiver_bytes is None else per_receiver_bytes * distinct,
                         rx["batched_ms"], "distinct (snapshot, receiver) walks",
                         "algorithmic bytes per receiver walk from the oracle's counts on the "
                         "single-snapshot field (same generator and parameters), times the "
                         "distinct walks done, over the batched time"),
        "rows_accounting": None if per_receiver_bytes is None else {
            "frac": per_receiver_bytes * total / (rx["batched_ms"] * 1e-3) / 1e9 / hbm_peak,
            "note": "every row counted as its own walk, although only the distinct ones are "
                    "walked and the rest are copied: not a memory roofline"},
        "bucket": {
            "flags": "TREVR2_BUCKET (per-bucket beams, the paper's scheme; the plain arm is "
                     "trevr2_J with TREVR2_BUCKET per subset)",
            "distinct_buckets": int(buckets), "plain_bucket_walks": int(plain_bucket_walks),
            **bk,
            "batched_units_per_s": units / (bk["batched_ms"] * 1e-3),
            "plain_units_per_s": units / (bk["plain_ms"] * 1e-3),
            "roofline": roof(None if per_bucket_walk_bytes is None else
                             per_bucket_walk_bytes * buckets + per_receiver_eval_bytes * distinct,
                             bk["batched_ms"],
                             "distinct (snapshot, bucket) walks + distinct receivers evaluated",
                             "algorithmic bytes of a bucket walk from the oracle's per-bucket "
                             "counts, plus per receiver one source record per source and its J "
                             "row"),
        },
    }
    for tr in trees:
        tr.free()
    return out


def run_adjoint(args, dev):
    """Adjoint cost: the 64^3 lognormal field (sigma 1), 1024 sources, 2 bands,
    nside 2, theta 0.75, every gas element a receiver, Loss = sum_i w_i J_i
    with w ~ U(0,1).  Forward = the J walk; backward = trevr2_J_backward
    (adjoint walk, table adjoint, element sums); tree and tables are built
    once before timing."""
    import torch

    import paper_2310_15235_gb300 as t2

    case = workloads.adjoint_case()
    nside, theta = case["nside"], case["theta"]
    d = {k: torch.from_numpy(np.ascontiguousarray(case[k])).to(dev)
         for k in ("pos", "mass", "kappa", "lum", "h", "active")}
    tree = t2.build(d["pos"], d["mass"], d["kappa"], d["lum"], d["h"], case["box_lo"],
                    case["box_size"], case["bucket"], device=dev)
    tree.prepare(nside)
    A, nb = len(case["active"]), case["nb"]
    w = torch.rand((A, nb), device=dev, generator=torch.Generator(dev).manual_seed(5))
    J = torch.empty((A, nb), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    reps = 3

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        tree.status()
        return e0.elapsed_time(e1) / reps

    fwd = timed(lambda: tree.J(d["active"], nside, theta, out=J, flags=t2.ASYNC))
    bwd = timed(lambda: tree.J_backward(d["active"], w, nside, theta, flags=t2.ASYNC))
    units = A * 12 * nside ** 2 * nb
    tree.free()
    return {"workload": "64^3 lognormal gas (sigma 1.0) + 1024 sources, 2 bands, nside 2, "
                        "theta 0.75, all 262,144 gas receivers, Loss = sum_i w_i J_i",
            "forward_ms": fwd, "backward_ms": bwd, "ratio": bwd / fwd,
            "forward_units_per_s": units / (fwd * 1e-3),
            "backward_units_per_s": units / (bwd * 1e-3)}


def run_bucket(case, inp, dev, per_receiver_walk_ms, reps=3, extra_flags=0,
               kernel="k_walk_bucket"):
    """Per-bucket beams (TREVR2_BUCKET, plus extra_flags) on the benchmark
    field: the same J with one walk per leaf from its centre; tree and
    tables built once, one warm-up and `reps` timed walks."""
    import torch

    import paper_2310_15235_gb300 as t2

    tree = t2.build(inp["pos"], inp["mass"], inp["kappa"], inp["lum"], inp["h"], case["box_lo"],
                    case["box_size"], case["bucket"], device=dev)
    tree.prepare(case["nside"])
    A, nb, npix = len(case["active"]), case["nb"], 12 * case["nside"] ** 2
    J = torch.empty((A, nb), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    flags = t2.ASYNC | t2.BUCKET | extra_flags
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0.record(stream)
    tree.J(inp["active"], case["nside"], case["theta"], out=J, flags=flags)
    w1.record(stream)
    torch.cuda.synchronize()
    first_ms = w0.elapsed_time(w1)  # includes tables built on first use
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        tree.J(inp["active"], case["nside"], case["theta"], out=J, flags=flags)
    e1.record(stream)
    torch.cuda.synchronize()
    tree.status()
    ms = e0.elapsed_time(e1) / reps
    out = {"walk_ms": ms, "units_per_s": A * npix * nb / (ms * 1e-3), "unit": UNIT,
           "kernel": kernel, "flags": flags & ~t2.ASYNC, "first_call_ms": first_ms,
           "speedup_vs_per_receiver": per_receiver_walk_ms / ms,
           "_J": J.cpu().numpy()}
    tree.free()
    return out


def run_adjoint_clumpy(case, inp, dev):
    """Adjoint / forward on the benchmark field itself (2,097,152 receivers,
    nside 4, 3 bands), Loss = sum w J with w ~ U(0,1); one warm-up and two
    timed calls of each."""
    import torch

    import paper_2310_15235_gb300 as t2

    tree = t2.build(inp["pos"], inp["mass"], inp["kappa"], inp["lum"], inp["h"], case["box_lo"],
                    case["box_size"], case["bucket"], device=dev)
    tree.prepare(case["nside"])
    A, nb = len(case["active"]), case["nb"]
    w = torch.rand((A, nb), device=dev, generator=torch.Generator(dev).manual_seed(6))
    J = torch.empty((A, nb), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        tree.status()
        return e0.elapsed_time(e1) / reps

    fwd = timed(lambda: tree.J(inp["active"], case["nside"], case["theta"], out=J, flags=t2.ASYNC))
    bwd = timed(lambda: tree.J_backward(inp["active"], w, case["nside"], case["theta"],
                                        flags=t2.ASYNC))
    tree.free()
    return {"forward_ms": fwd, "backward_ms": bwd, "ratio": bwd / fwd}


def run_walk_only(args):
    """The walk kernel alone on a clumpy field of lattice^3 gas (profiling
    aid): tree and tables built once, then `warmup + steps` walks."""
    import torch

    import paper_2310_15235_gb300 as t2

    dev = torch.device("cuda", 0)
    n = args.lattice
    case = workloads._clumpy(1003, n, 1.5, max(1, 10_000 * n ** 3 // 128 ** 3), [10.0, 3.0, 0.5],
                             4, 0.5, f"clumpy_multiband_{n}")
    inp = {k: torch.from_numpy(np.ascontiguousarray(case[k])).to(dev)
           for k in ("pos", "mass", "kappa", "lum", "h", "active")}
    tree = t2.build(inp["pos"], inp["mass"], inp["kappa"], inp["lum"], inp["h"], case["box_lo"],
                    case["box_size"], case["bucket"], device=dev)
    tree.prepare(case["nside"])
    A, nb, npix = len(case["active"]), case["nb"], 12 * case["nside"] ** 2
    J = torch.empty((A, nb), dtype=torch.float32, device=dev)
    times = []
    for k in range(args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tree.J(inp["active"], case["nside"], case["theta"], out=J,
               flags=t2.ASYNC | (t2.BUCKET if args.bucket else 0)
               | (t2.BUCKET | t2.PP | t2.THICK if args.pp else 0)
               | (t2.BUCKET | t2.CSM if args.csm else 0))
        e1.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            times.append(e0.elapsed_time(e1))
    tree.status()
    ms = float(np.mean(times))
    print(json.dumps({"mode": "walk-only", "bucket": bool(args.bucket or args.pp or args.csm),
                      "pp": bool(args.pp), "csm": bool(args.csm), "lattice": n,
                      "receivers": A, "walk_ms": ms,
                      "units_per_s": A * npix * nb / (ms * 1e-3), "nodes": tree.n_nodes,
                      "max_depth": tree.max_depth}), flush=True)
    tree.free()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--reference-sample", type=int, default=2048)
    ap.add_argument("--walk-only", action="store_true",
                    help="time only the walk kernel on a lattice^3 clumpy field (profiling)")
    ap.add_argument("--lattice", type=int, default=128)
    ap.add_argument("--bucket", action="store_true",
                    help="with --walk-only: per-bucket beams (TREVR2_BUCKET)")
    ap.add_argument("--pp", action="store_true",
                    help="with --walk-only: per-bucket beams with p-p absorption and "
                         "TREVR2_THICK")
    ap.add_argument("--csm", action="store_true",
                    help="with --walk-only: per-bucket beams with the complex source model")
    ap.add_argument("--no-bucket", action="store_true",
                    help="skip the per-bucket beams measurement")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the individual-timestep batching measurement")
    ap.add_argument("--batched-reps", type=int, default=2)
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint / forward timing")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="time only the forward and adjoint walks on the 64^3 adjoint field "
                         "(profiling)")
    args = ap.parse_args()
    if args.walk_only:
        run_walk_only(args)
        return
    if args.adjoint_only:
        import torch
        print(json.dumps({"mode": "adjoint-only",
                          **run_adjoint(args, torch.device("cuda", 0))}), flush=True)
        return
    world, rank, local = _dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
