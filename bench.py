"""Benchmark: quantized-BVH neighbor list (build + query) plus the fused LJ
energy/force pass on the LJ fluid with N = 2,097,152 particles at rho = 0.8.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = qbvh_build + qbvh_query (with its overflow check) + the LJ
energy/force pass, all on the GPU; inputs are resident in HBM.  Between timed
steps L2 is flushed by writing a 256 MiB buffer (outside the timed events).
Timing: CUDA events per stage on the launching stream; max over ranks.

``--impl reference`` times the CPU oracle (cell list + FP64 LJ) on the host
cores for the same workload and metric; only rank 0 runs it.

With --gpus N > 1 (torchrun) every rank runs an independent replica of the
workload on its own GPU; value = all ranks' particles / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "nlist particles/s (build+query), LJ N=2M; batched vs per-system; E/F grad err"
WORKLOAD = "lj_n2097152_rho0.8"
R_CUT = 3.0
CAP = 256


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples (the JSON line carries their summary); QBVH_BENCH_OUT overrides the folder
        out_dir = os.environ.get("QBVH_BENCH_OUT", os.path.join(ROOT, "bench_out"))
        self.path = os.path.join(out_dir, f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "samples": len(sm), "reasons": sorted(reasons)}


# DRAM bytes (read + write) and warp instructions executed of one traversal launch at
# N = 2,097,152, measured with ncu (profiles/query_warp_kernel_lj_n2097152.md) for the
# options of each entry and the traversal sources whose SHA-256 prefix is given; any
# other source or options report null.
PROFILED_TRAFFIC = {
    "source_sha256": "ba179f7ae5a5ff5c",
    "entries": [
        {"options": {"bundle_k": 64, "node_format": 0, "traversal": 1, "warp_particles": 32, "query_block": 128,
                     "fused_lj": 0, "persistent": 0},
         "bytes": 109.72e6 + 1007.59e6, "warp_inst": 1336503549},
        {"options": {"bundle_k": 64, "node_format": 0, "traversal": 1, "warp_particles": 32, "query_block": 256,
                     "fused_lj": 0, "persistent": 0},
         "bytes": 108.79e6 + 1006.68e6, "warp_inst": 1336503581},
        {"options": {"bundle_k": 64, "node_format": 1, "traversal": 1, "warp_particles": 32, "query_block": 128,
                     "fused_lj": 0, "persistent": 0},
         "bytes": 107.69e6 + 994.58e6, "warp_inst": 1302335900},
        {"options": {"bundle_k": 64, "node_format": 1, "traversal": 1, "warp_particles": 32, "query_block": 256,
                     "fused_lj": 0, "persistent": 0},
         "bytes": 107.69e6 + 994.40e6, "warp_inst": 1302335932},
    ],
}
# kernels of one timed step: build = prepare, Morton (+ sort histograms), segment
# scan, 4 onesweep passes (30-bit keys, 8-bit digits), Karras, fit; query = 1
# traversal launch (all periodic images); LJ = forward + fixed-order FP64 finalize
KERNELS_PER_STEP = 9 + 1 + 2
# with the LJ terms summed inside the traversal: build, traversal, finalize
KERNELS_PER_STEP_FUSED = 9 + 1 + 1
_TRAFFIC_SOURCES = ("paper_1901_08088_gb300/csrc/query.cu", "paper_1901_08088_gb300/csrc/qbvh_internal.cuh")


def traversal_source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for rel in _TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_entry(opts: dict, n: int):
    try:
        sha = traversal_source_hash()
    except OSError:
        return None
    if n != 2_097_152 or sha != PROFILED_TRAFFIC["source_sha256"]:
        return None
    for e in PROFILED_TRAFFIC["entries"]:
        if all(opts.get(k) == v for k, v in e["options"].items()):
            return e
    return None


def _profiled_traffic(opts: dict, n: int):
    e = _profiled_entry(opts, n)
    return None if e is None else e["bytes"]


def _issue_roofline(opts: dict, n: int, query_ms: float, clocks):
    """The traversal's binding resource is instruction issue: warp instructions
    per launch (ncu, profiled options and sources only) over the live duration,
    against one instruction per cycle per scheduler (4 per SM) at the SM clock
    sampled during the timed region."""
    import torch

    e = _profiled_entry(opts, n)
    if e is None or "warp_inst" not in e or not clocks:
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = sms * 4 * clocks["sm_mhz"] * 1e6
    achieved = e["warp_inst"] / (query_ms * 1e-3)
    return {"bound": "issue", "unit": "warp instructions/s", "achieved": achieved, "peak": peak,
            "frac": achieved / peak, "warp_inst_per_launch": e["warp_inst"], "sms": sms,
            "schedulers_per_sm": 4, "sm_mhz": clocks["sm_mhz"]}


# keys printed last in the JSON line, most important at the very end, so that a
# reader who keeps only the tail of the output still sees them
_TAIL_KEYS = ("configs", "grid_comparison", "fp64_data", "false_positives_per_particle", "autotune",
              "node_formats", "cpu_baseline", "grad_err", "split_ms", "breakdown_ms", "batched",
              "nlist_particles_per_s")


def _tail_order(out: dict) -> dict:
    head = {k: v for k, v in out.items() if k not in _TAIL_KEYS}
    tail = {k: out[k] for k in _TAIL_KEYS if k in out}
    return {**head, **tail}


def max_over_ranks(x: float) -> float:
    """Largest value of x over the ranks of the default process group (x itself
    without one).  The tensor lives where the backend needs it: CUDA for NCCL,
    CPU for gloo."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _alg_bytes(n: int, total_neighbors: int) -> int:
    # positions read once (16 B), counts written (4 B), list entries written (4 B each)
    return 16 * n + 4 * n + 4 * int(total_neighbors)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import workloads
    from paper_1901_08088_gb300 import NeighborList, _lib, autotune
    from paper_1901_08088_gb300.qbvh import qbvh_lj_forward, check

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    if args.n:
        # smaller case of the same fluid (density, jitter, radius) for profiling only
        s = workloads.jittered_lattice(args.n, 0.8, 0.25, seed=rank, r_cut=3.0, skin=0.3)
    else:
        s = workloads.workload(WORKLOAD, seed=rank)
    n = s.n
    pos4_host = torch.from_numpy(workloads.pack_float4(s.pos, s.types)).pin_memory()
    pos4 = pos4_host.cuda()
    nl = NeighborList(local)
    eps = torch.ones((1, 1), dtype=torch.float32, device="cuda")
    sig = torch.ones((1, 1), dtype=torch.float32, device="cuda")
    U = torch.empty(1, dtype=torch.float64, device="cuda")
    F = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    rc = np.full((1, 1), R_CUT, np.float32)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # one step: build, then the traversal and the LJ energy/forces over its
    # list through qbvh_query_lj_async (LJ terms inside the traversal when
    # QBVH_OPT_FUSED_LJ = 1, else the traversal and the list pass back to back)
    def step(p4):
        nl.build(p4, s.L)
        nl.query_lj_async(p4, s.r_list, CAP, eps, sig, rc, None, U, F, None, None)

    # options: explicit flags win; otherwise the autotuner picks them during
    # warm-up (the paper tunes launch parameters at run time, then freezes them)
    explicit = {}
    if args.bundle:
        explicit[_lib.QBVH_OPT_BUNDLE] = args.bundle
    if args.block:
        explicit[_lib.QBVH_OPT_QUERY_BLOCK] = args.block
    if args.traversal >= 0:
        explicit[_lib.QBVH_OPT_TRAVERSAL] = args.traversal
    if args.node_format >= 0:
        explicit[_lib.QBVH_OPT_NODE_FORMAT] = args.node_format
    if args.warp_particles:
        explicit[_lib.QBVH_OPT_WARP_PARTICLES] = args.warp_particles
    if args.lj_lanes:
        explicit[_lib.QBVH_OPT_LJ_LANES] = args.lj_lanes
    if args.lj_zorder >= 0:
        explicit[_lib.QBVH_OPT_LJ_ZORDER] = args.lj_zorder
    if args.fused_lj >= 0:
        explicit[_lib.QBVH_OPT_FUSED_LJ] = args.fused_lj
    if args.persistent >= 0:
        explicit[_lib.QBVH_OPT_PERSISTENT] = args.persistent
    tuned, tune_evals = dict(explicit), 0
    if not args.no_autotune:
        def tune_step(opts):
            for k, v in opts.items():
                nl.set_option(k, v)
            step(pos4)
        full = dict(autotune.OPTION_SPACE)
        full[_lib.QBVH_OPT_FUSED_LJ] = autotune.OPTIONAL_SPACE[_lib.QBVH_OPT_FUSED_LJ]
        space = {k: v for k, v in full.items() if k not in explicit}
        tuned, _, log = autotune.tune(tune_step, space=space, start=explicit, reps=3, warmup=1, sweeps=2)
        tune_evals = len(log)
    for k, v in tuned.items():
        nl.set_option(k, v)

    for _ in range(args.warmup):
        step(pos4)
    torch.cuda.synchronize()
    rc_q, _ = nl.query_status()
    if rc_q != 0:
        raise RuntimeError(f"query failed in warm-up: {_lib.QBVHError(rc_q)}")
    fused = nl.get_option(_lib.QBVH_OPT_FUSED_LJ) == 1
    mean_nbrs = float(nl.neighbors()[1].double().mean().item())
    total_nbrs = int(nl.neighbors()[1].long().sum().item())

    stream = torch.cuda.current_stream()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        e0, e1, e2 = ev[k]
        e0.record(stream)
        nl.build(pos4, s.L)
        e1.record(stream)
        nl.query_lj_async(pos4, s.r_list, CAP, eps, sig, rc, None, U, F, None, None)
        e2.record(stream)
        # the query's status, once the step has run (outside the events): a
        # failed or overflowed query invalidates the step
        stream.synchronize()
        rc_q, mx = nl.query_status()
        if rc_q != 0:
            raise RuntimeError(f"query failed in timed step: {_lib.QBVHError(rc_q)}")
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    t_build = np.array([ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)])
    t_qlj = np.array([ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)])
    t_step = t_build + t_qlj
    total_ms = max_over_ranks(float(t_step.sum()))

    # the same options with the traversal and the list pass as two launches,
    # each timed on its own: the list's build + query time (the metric's
    # neighbor-list part) and the plain traversal's roofline
    def split_times(reps):
        nl.set_option(_lib.QBVH_OPT_FUSED_LJ, 0)
        for _ in range(3):
            step(pos4)
        tb, tq, tl = [], [], []
        for k in range(reps):
            flush.fill_(float(k))
            f = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            f[0].record(stream)
            nl.build(pos4, s.L)
            f[1].record(stream)
            nl.query_async(s.r_list, CAP)
            f[2].record(stream)
            check(qbvh_lj_forward(nl.h, pos4, eps, sig, rc, None, U, F, None, None), "lj")
            f[3].record(stream)
            f[3].synchronize()
            rc_q, _ = nl.query_status()
            if rc_q != 0:
                raise RuntimeError(f"query failed: {_lib.QBVHError(rc_q)}")
            tb.append(f[0].elapsed_time(f[1]))
            tq.append(f[1].elapsed_time(f[2]))
            tl.append(f[2].elapsed_time(f[3]))
        nl.set_option(_lib.QBVH_OPT_FUSED_LJ, 1 if fused else 0)
        return np.array(tb), np.array(tq), np.array(tl)

    s_build, t_query, t_lj = split_times(max(5, min(args.steps, 20)))

    # build and query under each node format (the tuned options otherwise):
    # the paper's 10-bit quantized nodes (Fig. 3b) and FP32 nodes (Fig. 3a)
    node_formats = {}
    fmt_now = nl.get_option(_lib.QBVH_OPT_NODE_FORMAT)
    for fmt, name in ((0, "quantized_10bit_16B"), (1, "fp32_32B"), (2, "quantized_21bit_32B")):
        nl.set_option(_lib.QBVH_OPT_NODE_FORMAT, fmt)
        for _ in range(3):
            step(pos4)
        tb, tq = [], []
        for k in range(max(5, min(args.steps, 20))):
            flush.fill_(float(k))
            f0, f1, f2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            f0.record(stream)
            nl.build(pos4, s.L)
            f1.record(stream)
            nl.query_async(s.r_list, CAP)
            f2.record(stream)
            f2.synchronize()
            rc_q, _ = nl.query_status()
            if rc_q != 0:
                raise RuntimeError(f"query failed: {_lib.QBVHError(rc_q)}")
            tb.append(f0.elapsed_time(f1))
            tq.append(f1.elapsed_time(f2))
        node_formats[name] = {"build_ms": float(np.median(tb)), "query_ms": float(np.median(tq)),
                              "nlist_particles_per_s": n / ((float(np.median(tb)) + float(np.median(tq))) * 1e-3)}
    nl.set_option(_lib.QBVH_OPT_NODE_FORMAT, fmt_now)
    step(pos4)
    torch.cuda.synchronize()

    # end-to-end through the public API with host buffers: every step copies
    # its positions host -> device and its forces and energy device -> host
    # inside the timed region.  The copies run on a second stream with double
    # buffers, so that step k's results and step k+1's inputs move while step
    # k computes.
    def step_io(p4, Fo, Uo):
        nl.build(p4, s.L)
        nl.query_lj_async(p4, s.r_list, CAP, eps, sig, rc, None, Uo, Fo, None, None)

    copy = torch.cuda.Stream()
    P = [pos4, torch.empty_like(pos4)]
    Fd = [F, torch.empty_like(F)]
    Ud = [U, torch.empty_like(U)]
    F_host = [torch.empty((n, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
    U_host = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    loaded = [torch.cuda.Event() for _ in range(2)]
    computed = [torch.cuda.Event() for _ in range(2)]
    e2e_steps = max(2, min(args.steps, 32))
    torch.cuda.synchronize()
    ee0 = torch.cuda.Event(enable_timing=True)
    ee1 = torch.cuda.Event(enable_timing=True)
    flush.fill_(0.0)
    ee0.record(stream)
    copy.wait_event(ee0)
    with torch.cuda.stream(copy):
        P[0].copy_(pos4_host, non_blocking=True)
        loaded[0].record(copy)
    for k in range(e2e_steps):
        b = k % 2
        if k + 1 < e2e_steps:
            nb = (k + 1) % 2
            with torch.cuda.stream(copy):
                if k >= 1:
                    copy.wait_event(computed[nb])   # step k-1 is done with P[nb], Fd[nb]
                P[nb].copy_(pos4_host, non_blocking=True)
                loaded[nb].record(copy)
        stream.wait_event(loaded[b])
        step_io(P[b], Fd[b], Ud[b])
        computed[b].record(stream)
        with torch.cuda.stream(copy):
            copy.wait_event(computed[b])
            F_host[b].copy_(Fd[b], non_blocking=True)
            U_host[b].copy_(Ud[b], non_blocking=True)
    stream.wait_stream(copy)
    ee1.record(stream)
    ee1.synchronize()
    e2e_ms = ee0.elapsed_time(ee1)
    last = (e2e_steps - 1) % 2
    # every step copies the same positions, so the last step's query status
    # stands for all of them
    rc_q, _ = nl.query_status()
    if rc_q != 0:
        raise RuntimeError(f"query failed in an end-to-end step: {_lib.QBVHError(rc_q)}")
    if not torch.equal(F_host[last], Fd[last].cpu()):
        raise RuntimeError("end-to-end forces differ from the device result")
    e2e_ms = max_over_ranks(e2e_ms)

    out = None
    if rank == 0:
        peaks = _peaks()
        hbm = float(peaks["hbm_gbs"]) if peaks else 6800.0
        peak_src = "measured" if peaks else "fallback"
        bytes_q = _alg_bytes(n, total_nbrs)
        opts_now = autotune.option_names({k: nl.get_option(k) for k in autotune.OPTION_SPACE})
        q_only = bytes_q / (float(t_query.mean()) * 1e-3) / 1e9
        nlist_ms = float(s_build.mean()) + float(t_query.mean())
        if fused:
            # the traversal also reads nothing more and writes the forces (12 B per particle)
            bytes_k = bytes_q + 12 * n
            achieved = bytes_k / (float(t_qlj.mean()) * 1e-3) / 1e9
            kname = ("query_warp_lj_kernel (traversal + exact leaf test + list write + LJ terms of the "
                     "accepted pairs; the timed stage includes the FP64 finalize)")
        else:
            bytes_k = bytes_q
            achieved = q_only
            kname = "query_warp_kernel (traversal + exact leaf test + list write)"
        step_alg = (bytes_q + 12 * n) / (float(t_step.mean()) * 1e-3) / 1e9
        value = world * n * args.steps / (total_ms * 1e-3)
        out = {
            "metric": METRIC,
            "value": value,
            "unit": "particles/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": "LJ fluid N=2,097,152 rho=0.8 jittered lattice (+-0.25), r_list=3.3, cap 256, "
                            "build+query+LJ energy/force (r_cut=3.0, eps=sig=1)",
                "n": n, "L": float(s.L), "r_list": float(s.r_list[0, 0]), "cap": CAP,
                "mean_neighbors": mean_nbrs,
                "l2": "flushed between timed steps (256 MiB write, outside the timed events)",
                "parallelism": f"replicas x{world}",
                "bundle_k": nl.get_option(_lib.QBVH_OPT_BUNDLE),
                "query_block": nl.get_option(_lib.QBVH_OPT_QUERY_BLOCK),
                "traversal": ["thread_per_particle", "warp_per_32_particles"][
                    nl.get_option(_lib.QBVH_OPT_TRAVERSAL)],
                "node_format": ["quantized_10bit_16B", "fp32_32B", "quantized_21bit_32B"][
                    nl.get_option(_lib.QBVH_OPT_NODE_FORMAT)],
                "lj_lanes_per_particle": nl.get_option(_lib.QBVH_OPT_LJ_LANES),
            },
            "breakdown_ms": {"build": float(t_build.mean()), "query_lj": float(t_qlj.mean()),
                             "fused_lj": fused},
            "split_ms": {"build": float(s_build.mean()), "query": float(t_query.mean()),
                         "lj": float(t_lj.mean()),
                         "note": "the same options with the traversal and the LJ list pass as two launches"},
            "node_formats": node_formats,
            "nlist_particles_per_s": n / (nlist_ms * 1e-3),
            "roofline": {
                "kernel": kname,
                "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm,
                "traffic": _profiled_traffic(dict(opts_now, fused_lj=int(fused)), n),
                "peak_source": peak_src,
                "alg_bytes_per_launch": bytes_k,
                "step_frac": step_alg / hbm,
                "query_only": {"kernel": "query_warp_kernel (traversal + exact leaf test + list write)",
                               "query_ms": float(t_query.mean()), "alg_bytes_per_launch": bytes_q,
                               "achieved": q_only, "frac": q_only / hbm,
                               "traffic": _profiled_traffic(dict(opts_now, fused_lj=0), n),
                               "issue": _issue_roofline(dict(opts_now, fused_lj=0), n, float(t_query.mean()),
                                                        clocks)},
            },
            "e2e": {"value": world * n * e2e_steps / (e2e_ms * 1e-3), "unit": "particles/s",
                    "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 12 * n + 8,
                    "steps": e2e_steps, "ms_per_step": e2e_ms / e2e_steps,
                    "copies": "second stream, double-buffered: step k's D2H and step k+1's H2D overlap step k",
                    "l2": "not flushed; every step writes and reads its 1 GB list, larger than L2"},
            "gpu_launches": args.steps * (KERNELS_PER_STEP_FUSED if fused else KERNELS_PER_STEP),
            "autotune": {"evaluations": tune_evals, "chosen": autotune.option_names(
                {k: nl.get_option(k) for k in autotune.OPTION_SPACE})},
            "clocks": clocks,
            "wall_s_timed": wall,
        }
        if args.n:
            out["config"]["workload"] = f"profiling case: LJ fluid N={n} rho=0.8 (not a bench result)"
        if not args.no_batched and world == 1:
            out["batched"] = run_batched(args, local)
        if not args.no_grid_compare and world == 1 and not args.n:
            out["grid_comparison"] = run_grid_comparison(args, local)
            out["fp64_data"] = run_fp64_comparison(args, local)
            out["false_positives_per_particle"] = run_false_positives(local)
            out["configs"] = run_configs(args, local, hbm, nlist_ms, mean_nbrs,
                                         out.get("batched"), {k: nl.get_option(k) for k in autotune.OPTION_SPACE})
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline(s, samples=1)
            if not args.n:
                out["grad_err"] = gradient_check(local)
                if out.get("configs"):
                    cpu_configs(out["configs"])
        elif world == 1:
            out["cpu_baseline"] = None
    nl.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


def run_batched(args, local):
    """256 independent systems: batched build+query from one CUDA graph vs the per-system loop."""
    import torch

    import workloads
    from paper_1901_08088_gb300 import BatchedNeighborList, PerSystemLoop, _lib, autotune

    systems = workloads.workload("ensemble_256", seed=0)
    pos4 = np.concatenate([workloads.pack_float4(x.pos, x.types) for x in systems])
    off = np.concatenate([[0], np.cumsum([x.n for x in systems])]).astype(np.int32)
    Ls = np.array([x.L for x in systems], np.float32)
    total = int(off[-1])
    buf = torch.from_numpy(pos4).cuda()
    r = systems[0].r_list
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    runners = {}

    def graph_step(opts):
        key = tuple(sorted(opts.items()))
        if key not in runners:
            runners[key] = BatchedNeighborList(buf, off, Ls, r, cap=128, options=opts, device=local).capture()
        g = runners[key]
        g.replay()

    space = {k: autotune.OPTION_SPACE[k] for k in (_lib.QBVH_OPT_BUNDLE, _lib.QBVH_OPT_NODE_FORMAT,
                                                   _lib.QBVH_OPT_QUERY_BLOCK, _lib.QBVH_OPT_PERSISTENT)}
    space[_lib.QBVH_OPT_WARP_PARTICLES] = [32, 16, 8]
    best, _, _ = autotune.tune(graph_step, space=space, reps=3, warmup=1, sweeps=1)
    g = runners[tuple(sorted(best.items()))]
    for x in runners.values():
        if x is not g:
            x.close()
    for _ in range(3):
        assert g.run() == _lib.QBVH_OK
    reps = max(args.steps, 5)
    graph_ms = timed(lambda: (g.replay(), stream.synchronize(), g.status()), reps)
    # the same batched launches issued eagerly: what the graph saves in launch overhead
    eager_ms = timed(lambda: (g.enqueue_eager(), stream.synchronize(), g.status()), reps)
    loop = PerSystemLoop(buf, off, Ls, r, cap=g.cap, options=best, device=local)
    for _ in range(2):
        assert loop.run() == _lib.QBVH_OK
    loop_ms = timed(lambda: loop.run(), reps)
    loop.close()
    g.close()
    return {
        "workload": f"{len(systems)} LJ systems, N log-uniform [500, 50000] (sum N = {total}), "
                    "rho U[0.3, 0.9], jitter 0.3, r_list = 2.8; build + query per step",
        "graph_particles_per_s": total / (graph_ms * 1e-3),
        "loop_particles_per_s": total / (loop_ms * 1e-3),
        "graph_ms": graph_ms, "loop_ms": loop_ms, "ratio": loop_ms / graph_ms,
        "eager_batched_ms": eager_ms, "eager_batched_particles_per_s": total / (eager_ms * 1e-3),
        "options": autotune.option_names(best),
    }


def run_grid_comparison(args, local):
    """The paper's comparison (Sec. 4): quantized BVH vs an equivalent sort-based
    uniform grid, build + query of the exact list, on synthetic stand-ins of its
    LJ state points (N = 128,000, r_c = 3.0, rho 0.2 and 0.8; N scan at rho 0.6)
    and on the bench workload.  Each method gets a small autotune."""
    import torch

    import workloads
    from paper_1901_08088_gb300 import NeighborList, _lib, autotune

    cases = [("paper LJ rho 0.2", 128_000, 0.2, 3.0, 0.0), ("paper LJ rho 0.8", 128_000, 0.8, 3.0, 0.0)]
    cases += [("paper WCA rho 0.2", 128_000, 0.2, workloads.WCA_RCUT, 0.0),
              ("paper WCA rho 0.8", 128_000, 0.8, workloads.WCA_RCUT, 0.0)]
    cases += [(f"N scan rho 0.6", n, 0.6, 3.0, 0.0) for n in (1_000, 4_096, 16_384, 65_536)]
    cases += [("spinodal-like liquid/vapor", 1_000_000, 0.2, 3.0, 0.0)]
    cases += [("bench workload", 2_097_152, 0.8, 3.0, 0.3)]
    out = []
    for label, n, rho, rc, skin in cases:
        if label.startswith("spinodal"):
            s = workloads.spinodal_like(n, rho, seed=0, r_cut=rc, skin=skin)
        else:
            # WCA: liquid-like disorder (jitter half the lattice spacing), so that
            # the short cutoff sees neighbors at rho 0.2 too
            jit = 0.25 if n == 2_097_152 else (0.5 * (1.0 / rho) ** (1.0 / 3.0) if "WCA" in label else 0.3)
            s = workloads.jittered_lattice(n, rho, jit, seed=0, r_cut=rc, skin=skin)
        pos4 = torch.from_numpy(workloads.pack_float4(s.pos, s.types)).cuda()
        res = {"workload": label, "n": n, "rho": rho, "r_list": float(s.r_list[0, 0])}
        for method, space in ((0, {_lib.QBVH_OPT_WARP_PARTICLES: [32, 16, 8, 4, 1],
                                    _lib.QBVH_OPT_BUNDLE: [8, 16, 32, 64], _lib.QBVH_OPT_NODE_FORMAT: [0, 1]}),
                              (1, {_lib.QBVH_OPT_GRID_LANES: [2, 4, 8, 16]})):
            nl = NeighborList(local)
            nl.set_option(_lib.QBVH_OPT_METHOD, method)

            def step(opts, nl=nl, pos4=pos4, s=s):
                for k, v in opts.items():
                    nl.set_option(k, v)
                nl.build(pos4, s.L)
                nl.query(s.r_list, cap=CAP)

            start = {k: v[0] for k, v in space.items()}
            best, ms, _ = autotune.tune(step, space=space, start=start, reps=5, warmup=2, sweeps=1)
            tag = "bvh" if method == 0 else "grid"
            res[f"{tag}_ms"] = ms
            res[f"{tag}_options"] = autotune.option_names(best)
            # split: build alone, then query alone (async enqueue + one wait)
            for k, v in best.items():
                nl.set_option(k, v)
            res[f"{tag}_build_ms"] = autotune.time_step(lambda o: nl.build(pos4, s.L), {}, reps=5, warmup=2)
            nl.build(pos4, s.L)
            res[f"{tag}_query_ms"] = autotune.time_step(lambda o: nl.query_async(s.r_list, CAP), {}, reps=5,
                                                        warmup=2)
            nl.close()
        res["bvh_speedup_over_grid"] = res["grid_ms"] / res["bvh_ms"]
        out.append(res)
    return out


def run_false_positives(local):
    """Alg. 1 without the exact leaf test (candidate mode) on the paper's LJ
    state points (N = 128,000, r_c = 3.0, rho 0.2 and 0.8; Sec. 4.1 counts the
    false positives of its 10-bit tree): false positives per particle with
    the leaves tested at each node format's precision -- 10-bit and 21-bit
    quantized boxes, and the FP32 points (the bit width Sec. 2.2 weighs)."""
    import torch

    import workloads
    from paper_1901_08088_gb300 import NeighborList, _lib

    out = {"paper": "about 1.5 and 3.8 false positives per particle at rho 0.2 and 0.8 with 10-bit nodes "
                    "(Sec. 4.1)"}
    for rho in (0.2, 0.8):
        s = workloads.jittered_lattice(128_000, rho, 0.3, seed=1, r_cut=3.0, skin=0.0)
        pos4 = torch.from_numpy(workloads.pack_float4(s.pos, s.types)).cuda()
        res = {}
        for fmt, name in ((0, "quantized_10bit"), (2, "quantized_21bit"), (1, "fp32")):
            counts = []
            for cand in (0, 1):
                nl = NeighborList(local)
                nl.set_option(_lib.QBVH_OPT_NODE_FORMAT, fmt)
                nl.set_option(_lib.QBVH_OPT_CANDIDATES, cand)
                nl.build(pos4, s.L)
                nl.query(s.r_list, cap=512)
                counts.append(float(nl.neighbors()[1].double().mean().item()))
                nl.close()
            res["true_neighbours"] = counts[0]
            res[name] = counts[1] - counts[0]
        out[f"rho_{rho}"] = res
    return out


def run_fp64_comparison(args, local):
    """Double-precision particle data (Sec. 2.2; the paper's double-precision
    benchmarks, Sec. 4.1-4.2): build + query of the exact FP64 list against the
    same positions rounded to FP32, on the LJ and WCA state points (N = 128,000,
    rho 0.2 / 0.8) and the bench workload.  Each gets a small autotune."""
    import torch

    import workloads
    from paper_1901_08088_gb300 import NeighborList, _lib, autotune

    half = lambda rho: 0.5 * (1.0 / rho) ** (1.0 / 3.0)   # liquid-like disorder for WCA
    cases = [("LJ rho 0.2", 128_000, 0.2, 3.0, 0.0, 0.3), ("LJ rho 0.8", 128_000, 0.8, 3.0, 0.0, 0.3),
             ("WCA rho 0.2", 128_000, 0.2, workloads.WCA_RCUT, 0.0, half(0.2)),
             ("WCA rho 0.8", 128_000, 0.8, workloads.WCA_RCUT, 0.0, half(0.8)),
             ("spinodal-like liquid/vapor", 1_000_000, 0.2, 3.0, 0.0, None),
             ("bench workload", 2_097_152, 0.8, 3.0, 0.3, 0.25)]
    space = {_lib.QBVH_OPT_BUNDLE: [64, 32, 16], _lib.QBVH_OPT_NODE_FORMAT: [0, 1]}
    out = []
    for label, n, rho, rc, skin, jit in cases:
        if jit is None:
            s64 = workloads.spinodal_like(n, rho, seed=0, r_cut=rc, skin=skin, double=True)
        else:
            s64 = workloads.jittered_lattice64(n, rho, jit, seed=0, r_cut=rc, skin=skin)
        L32 = np.float32(s64.L)
        p32 = s64.pos.astype(np.float32)
        p32[p32 >= L32] = 0.0
        pos4d = torch.from_numpy(workloads.pack_double4(s64.pos, s64.types)).cuda()
        pos4 = torch.from_numpy(workloads.pack_float4(p32, s64.types)).cuda()
        res = {"workload": label, "n": n, "rho": rho, "r_list": float(s64.r_list[0, 0])}
        for tag, build in (("fp64", lambda nl: nl.build_f64(pos4d, s64.L)),
                           ("fp32", lambda nl: nl.build(pos4, L32))):
            nl = NeighborList(local)

            def step(opts, nl=nl, build=build):
                for k, v in opts.items():
                    nl.set_option(k, v)
                build(nl)
                nl.query(s64.r_list, cap=CAP)

            best, ms, _ = autotune.tune(step, space=space, start={k: v[0] for k, v in space.items()},
                                        reps=5, warmup=2, sweeps=1)
            res[f"{tag}_ms"] = ms
            res[f"{tag}_options"] = autotune.option_names(best)
            res[f"{tag}_mean_neighbors"] = float(nl.neighbors()[1].float().mean().item())
            nl.close()
        res["fp64_over_fp32_time"] = res["fp64_ms"] / res["fp32_ms"]
        out.append(res)
    return out


def _config_systems(name):
    """The systems of one of the five configurations (a list; one entry unless batched)."""
    import workloads

    w = workloads.workload(name, seed=0)
    return w if isinstance(w, list) else [w]


CONFIG_NAMES = ["lj_n4096_rho0.6", "lj_n2097152_rho0.8", "mixture_L100", "ensemble_256", "lj2type_32x65536"]


def run_configs(args, local, hbm, bench_ms, bench_nbrs, batched, options):
    """Build + query of each of the five configurations on the GPU: particles/s
    and the fraction of the HBM roofline of its algorithmic bytes (16 N + 4 N +
    4 sum n_i).  Configuration 2 is the bench step's own build + query and
    configuration 4 the batched graph measured above; the others are timed here
    (one batched build for several systems), best of 10 after 3 warm-ups, after
    a small autotune that starts from the bench step's choice."""
    import torch

    import workloads
    from paper_1901_08088_gb300 import NeighborList, _lib, autotune

    out = []
    stream = torch.cuda.current_stream()
    for name in CONFIG_NAMES:
        systems = _config_systems(name)
        total = sum(q.n for q in systems)
        res = {"name": name, "n": total, "systems": len(systems)}
        if name == "lj_n2097152_rho0.8":
            ms = bench_ms
            res["mean_neighbors"] = float(bench_nbrs)
        elif name == "ensemble_256" and batched:
            ms = batched["graph_ms"]
        else:
            q0 = systems[0]
            pos4 = torch.from_numpy(np.concatenate([workloads.pack_float4(q.pos, q.types) for q in systems])).cuda()
            off = np.concatenate([[0], np.cumsum([q.n for q in systems])]).astype(np.int32)
            Ls = np.array([q.L for q in systems], np.float32)
            nl = NeighborList(local)
            cap = 512 if q0.n_types > 1 and name == "mixture_L100" else CAP

            def step(opts=None):
                for k, v in (opts or {}).items():
                    nl.set_option(k, v)
                if len(systems) == 1:
                    nl.build(pos4, q0.L, q0.n_types)
                else:
                    nl.build_batched(pos4, off, Ls, n_types=q0.n_types)
                nl.query(q0.r_list, cap=cap)

            # a small autotune per configuration, from the bench step's choice
            space = {_lib.QBVH_OPT_WARP_PARTICLES: [32, 16, 8, 4, 1], _lib.QBVH_OPT_BUNDLE: [16, 32, 64],
                     _lib.QBVH_OPT_NODE_FORMAT: [1, 0], _lib.QBVH_OPT_QUERY_BLOCK: [256, 128, 64]}
            if q0.n_types > 1 and np.all(np.asarray(q0.r_list) == np.asarray(q0.r_list).flat[0]):
                # one radius for every type pair: one tree per system is an option
                space[_lib.QBVH_OPT_TYPE_TREES] = autotune.OPTIONAL_SPACE[_lib.QBVH_OPT_TYPE_TREES]
            best, _, _ = autotune.tune(step, space=space, start=dict(options), reps=3, warmup=1, sweeps=1)
            res["options"] = autotune.option_names(best)
            step(best)
            for _ in range(2):
                step()
            ts = []
            for _ in range(10):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step()
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            ms = float(min(ts))
            res["mean_neighbors"] = float(nl.neighbors()[1].float().mean().item())
            nl.close()
            if len(systems) == 1 and total <= 65536:
                # a small system is bound by launch latency: the same build +
                # query replayed from a CUDA graph (BatchedNeighborList, one system)
                from paper_1901_08088_gb300 import BatchedNeighborList

                bl = BatchedNeighborList(pos4, off, Ls, q0.r_list, n_types=q0.n_types, cap=cap,
                                         options=best, device=local).capture()
                for _ in range(3):
                    bl.replay()
                reps = 50
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(reps):
                    bl.replay()
                b.record(stream)
                b.synchronize()
                if bl.status() == _lib.QBVH_OK:
                    res["graph_ms"] = a.elapsed_time(b) / reps
                    res["graph_particles_per_s"] = total / (res["graph_ms"] * 1e-3)
                bl.close()
        res["gpu_ms"] = ms
        res["gpu_particles_per_s"] = total / (ms * 1e-3)
        if "mean_neighbors" in res:
            alg = 20 * total + 4 * res["mean_neighbors"] * total
            res["hbm_frac"] = alg / (ms * 1e-3) / 1e9 / hbm
        out.append(res)
    return out


def cpu_configs(configs):
    """The oracle's cell list (build + query) on the five configurations: all
    host cores on the full configuration, and one thread (a child process with
    OMP_NUM_THREADS=1) on a bounded sample of it."""
    import oracle

    samples = {"lj_n4096_rho0.6": 1, "lj_n2097152_rho0.8": 1, "mixture_L100": 1, "ensemble_256": 16,
               "lj2type_32x65536": 2}
    for res in configs:
        systems = _config_systems(res["name"])
        t0 = time.perf_counter()
        for q in systems:
            oracle.nlist(q.pos, q.L, q.r_list, q.types, q.n_types, cap=512)
        res["cpu_all_cores_particles_per_s"] = res["n"] / (time.perf_counter() - t0)
        res["cpu_cores"] = oracle.num_threads()
        k = samples[res["name"]]
        code = (
            "import sys, time, numpy as np; sys.path.insert(0, %r); import oracle, workloads\n"
            "w = workloads.workload(%r, seed=0); w = w if isinstance(w, list) else [w]; w = w[:%d]\n"
            "if %r == 'lj_n2097152_rho0.8': w = [workloads.jittered_lattice(131072, 0.8, 0.25, 0, 3.0, 0.3)]\n"
            "t0 = time.perf_counter()\n"
            "for q in w: oracle.nlist(q.pos, q.L, q.r_list, q.types, q.n_types, cap=512)\n"
            "print(sum(q.n for q in w), time.perf_counter() - t0)\n") % (ROOT, res["name"], k, res["name"])
        env = dict(os.environ, OMP_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        try:
            nn, tt = r.stdout.split()[-2:]
            res["cpu_1thread_particles_per_s"] = float(nn) / float(tt)
            res["cpu_1thread_sample_particles"] = int(nn)
        except ValueError:
            res["cpu_1thread_particles_per_s"] = None


def gradient_check(local):
    """The differentiable LJ layer on its workload (Eq. 1 with per-type-pair
    eps / sigma, two types, 32 systems x 65,536 particles, one batched build +
    query): energies, forces and dU/deps, dU/dsigma through the autograd
    wrapper, against the FP64 oracle on the oracle's own lists.  Part of the
    CPU-baseline leg, the one bench leg that runs the oracle; also times the
    GPU forward + backward (build and query included)."""
    import torch

    import oracle
    import workloads
    from paper_1901_08088_gb300 import NeighborList, _lib, lj_energy

    systems = workloads.workload("lj2type_32x65536", seed=0)
    E, S = systems[0].meta["eps"], systems[0].meta["sig"]
    rc = 2.5
    pos4 = torch.from_numpy(np.concatenate([workloads.pack_float4(q.pos, q.types) for q in systems])).cuda()
    off = np.concatenate([[0], np.cumsum([q.n for q in systems])]).astype(np.int32)
    Ls = np.array([q.L for q in systems], np.float32)
    xyz = torch.from_numpy(np.concatenate([q.pos for q in systems])).cuda().requires_grad_(True)
    eps = torch.tensor(E, dtype=torch.float32, device="cuda", requires_grad=True)
    sig = torch.tensor(S, dtype=torch.float32, device="cuda", requires_grad=True)
    nl = NeighborList(local)
    # one list radius for both type pairs: one tree per system holds both types
    nl.set_option(_lib.QBVH_OPT_TYPE_TREES, 0)

    def fwd_bwd():
        for t in (xyz, eps, sig):
            t.grad = None
        nl.build_batched(pos4, off, Ls, n_types=2)
        nl.query(float(systems[0].r_list[0, 0]), cap=CAP)
        U = lj_energy(nl, xyz, eps, sig, rc, pos4=pos4)
        U.sum().backward()
        return U

    for _ in range(2):
        fwd_bwd()
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    a.record(stream)
    for _ in range(reps):
        U = fwd_bwd()
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    U = U.detach().cpu().numpy()
    gx = xyz.grad.cpu().numpy()
    ge, gs = eps.grad.cpu().numpy(), sig.grad.cpu().numpy()
    nl.close()
    worst_u = worst_f = 0.0
    dE = np.zeros((2, 2))
    dS = np.zeros((2, 2))
    for k, q in enumerate(systems):
        ro, co = oracle.nlist(q.pos, q.L, q.r_list, q.types, q.n_types)
        ref = oracle.lj_fp64(q.pos, q.types, q.L, E, S, np.float32(rc), ro, co)
        lo, hi = off[k], off[k + 1]
        worst_u = max(worst_u, abs(U[k] - ref["U"]) / abs(ref["U"]))
        worst_f = max(worst_f, float(np.linalg.norm(-gx[lo:hi] - ref["F"]) / np.linalg.norm(ref["F"])))
        dE += ref["dE"]
        dS += ref["dS"]
    return {"workload": "32 LJ systems x 65,536, two types, eps/sigma per type pair, r_cut 2.5, r_list 2.8",
            "reference": "FP64 oracle on its own lists",
            "U_rel_max": worst_u, "F_rel_max": worst_f,
            "dU_deps_rel_max": float(np.max(np.abs(ge - dE) / np.abs(dE))),
            "dU_dsigma_rel_max": float(np.max(np.abs(gs - dS) / np.abs(dS))),
            "tolerance": 1e-5, "forward_backward_ms": ms,
            "forward_backward_particles_per_s": float(off[-1]) / (ms * 1e-3)}


def cpu_baseline(s, samples=1):
    """The oracle as it stands: OpenMP cell list build+query + FP64 LJ, on the host cores."""
    import oracle

    t = []
    for _ in range(samples):
        t0 = time.perf_counter()
        rows, counts = oracle.nlist(s.pos, s.L, s.r_list, cap=CAP, method="cell")
        oracle.lj_fp64(s.pos, s.types, s.L, [[1.0]], [[1.0]], np.float32(R_CUT), rows, counts)
        t.append(time.perf_counter() - t0)
    tm = float(np.median(t))
    return {"value": s.n / tm, "unit": "particles/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{samples} full step(s) of the N={s.n} workload: cell-list build+query on "
                      f"{oracle.num_threads()} OpenMP threads, then the FP64 LJ energy/forces single-threaded "
                      f"(the oracle's LJ has no parallel loop); {tm:.2f} s per step"}


def reference_sample_n(steps: int, warmup: int) -> int:
    """Particles per reference step: 262,144 for runs of up to 256 steps, fewer
    for longer runs, so that the whole run stays within a few minutes."""
    k = steps + warmup
    return 262_144 if k <= 256 else (65_536 if k <= 1024 else 16_384)


def run_reference(args):
    """The CPU oracle as it stands, on the host cores (rank 0 only).

    Each step is a bounded sample of the workload: the same fluid (rho 0.8,
    jitter 0.25, r_list 3.3, r_cut 3.0) with N = 262,144 particles instead of
    2,097,152, so that a run with a large --steps count ends within minutes;
    the metric is a rate (particles/s), which the sample estimates (the sample
    shrinks further for very long runs, see reference_sample_n).
    """
    world, rank, _ = _dist()
    if rank != 0:
        return None
    import oracle
    import workloads

    oracle.build()
    s = workloads.jittered_lattice(reference_sample_n(args.steps, args.warmup), 0.8, 0.25, seed=0,
                                   r_cut=3.0, skin=0.3)

    def one():
        rows, counts = oracle.nlist(s.pos, s.L, s.r_list, cap=CAP, method="cell")
        oracle.lj_fp64(s.pos, s.types, s.L, [[1.0]], [[1.0]], np.float32(R_CUT), rows, counts)

    for _ in range(args.warmup):
        one()
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        one()
        t.append(time.perf_counter() - t0)
    total = float(np.sum(t))
    value = s.n * args.steps / total
    sample = (f"each of {args.steps} steps: the same fluid at N={s.n} (of the 2,097,152-particle workload): "
              f"cell-list build+query (OpenMP) + FP64 LJ energy/forces (1 thread); {total / args.steps:.3f} s/step")
    return {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "LJ fluid rho=0.8 jittered lattice (+-0.25), r_list=3.3, cap 256, "
                               f"build+query+LJ energy/force (r_cut=3.0); CPU oracle on a {s.n}-particle sample"},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-system graph-vs-loop measurement")
    ap.add_argument("--no-grid-compare", action="store_true", help="skip the BVH-vs-grid comparison")
    ap.add_argument("--n", type=int, default=0,
                    help="profiling aid: run the same fluid with N particles instead of 2,097,152 "
                         "(the line it prints is not a bench result)")
    ap.add_argument("--bundle", type=int, default=0, help="subtree-collapse size K (0: library default)")
    ap.add_argument("--block", type=int, default=0, help="traversal threads per block (0: library default)")
    ap.add_argument("--lj-lanes", type=int, default=0, help="lanes per particle in the LJ pass (0: default)")
    ap.add_argument("--lj-zorder", type=int, default=-1, help="LJ pass in Z-order (1) or original order (0)")
    ap.add_argument("--warp-particles", type=int, default=0, help="particles per warp of the walk (0: default)")
    ap.add_argument("--node-format", type=int, default=-1,
                    help="0: 10-bit quantized nodes, 1: FP32 nodes (-1: library default)")
    ap.add_argument("--persistent", type=int, default=-1,
                    help="traversal warps take packets from a queue (1) or one packet per warp (0); -1: autotuned")
    ap.add_argument("--fused-lj", type=int, default=-1,
                    help="LJ terms inside the traversal (1) or a separate list pass (0); -1: autotuned")
    ap.add_argument("--traversal", type=int, default=-1,
                    help="0: one thread per particle, 1: one warp per 32 particles (-1: library default)")
    args = ap.parse_args()
    if args.impl == "reference":
        out = run_reference(args)
    else:
        out = run_ours(args)
    if out is not None:
        print(json.dumps(_tail_order(out)), flush=True)


if __name__ == "__main__":
    main()
