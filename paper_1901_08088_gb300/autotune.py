"""Runtime autotuner for the launch and layout options.

The paper lets runtime autotuners pick the kernel launch parameters during
warm-up and then freezes them (Sec. 4).  Here the tuned options are the
subtree-collapse size, the node format (10-bit or 21-bit quantized, or FP32
bounds: the bit width of the quantization, Sec. 2.2), the
traversal mapping (thread or warp per particle), the traversal block size,
whether traversal warps take packets from a queue, and the lanes per particle
of the LJ pass; where every type pair has the same
list radius a caller may add one tree per system instead of one per type.
The search is coordinate descent:
each option in turn is swept with the others held at the best values so far,
for a fixed number of sweeps; every candidate is timed with CUDA events on
the current stream, best of ``reps`` runs after ``warmup`` runs.
"""
from __future__ import annotations

import json
import os

import torch

from . import _lib

__all__ = ["OPTION_SPACE", "OPTIONAL_SPACE", "DEFAULTS", "tune", "time_step", "option_names"]

OPTION_SPACE = {
    _lib.QBVH_OPT_BUNDLE: [8, 16, 32, 64],
    _lib.QBVH_OPT_NODE_FORMAT: [0, 1, 2],
    _lib.QBVH_OPT_TRAVERSAL: [1, 0],
    _lib.QBVH_OPT_WARP_PARTICLES: [32, 16, 8, 4, 1],
    _lib.QBVH_OPT_QUERY_BLOCK: [64, 128, 256],
    _lib.QBVH_OPT_LJ_LANES: [1, 2, 4, 8],
    _lib.QBVH_OPT_PERSISTENT: [0, 1],
}

# options a caller adds to the search where they apply: one tree per system
# only when every type pair has the same list radius; the LJ terms inside the
# traversal only for a step that evaluates LJ over the list it builds
OPTIONAL_SPACE = {
    _lib.QBVH_OPT_TYPE_TREES: [1, 0],
    _lib.QBVH_OPT_FUSED_LJ: [1, 0],
}

DEFAULTS = {
    _lib.QBVH_OPT_BUNDLE: 16,
    _lib.QBVH_OPT_NODE_FORMAT: 0,
    _lib.QBVH_OPT_TRAVERSAL: 1,
    _lib.QBVH_OPT_WARP_PARTICLES: 32,
    _lib.QBVH_OPT_QUERY_BLOCK: 128,
    _lib.QBVH_OPT_LJ_LANES: 2,
    _lib.QBVH_OPT_TYPE_TREES: 1,
    _lib.QBVH_OPT_FUSED_LJ: 0,
    _lib.QBVH_OPT_PERSISTENT: 0,
}

_NAMES = {
    _lib.QBVH_OPT_BUNDLE: "bundle_k",
    _lib.QBVH_OPT_NODE_FORMAT: "node_format",
    _lib.QBVH_OPT_TRAVERSAL: "traversal",
    _lib.QBVH_OPT_QUERY_BLOCK: "query_block",
    _lib.QBVH_OPT_LJ_LANES: "lj_lanes",
    _lib.QBVH_OPT_WARP_PARTICLES: "warp_particles",
    _lib.QBVH_OPT_GRID_LANES: "grid_lanes",
    _lib.QBVH_OPT_METHOD: "method",
    _lib.QBVH_OPT_LJ_ZORDER: "lj_zorder",
    _lib.QBVH_OPT_TYPE_TREES: "type_trees",
    _lib.QBVH_OPT_FUSED_LJ: "fused_lj",
    _lib.QBVH_OPT_PERSISTENT: "persistent",
}


def option_names(opts: dict) -> dict:
    return {_NAMES.get(k, str(k)): v for k, v in opts.items()}


def time_step(step, options: dict, reps: int = 5, warmup: int = 2) -> float:
    """Best time in ms of ``step(options)`` (which enqueues work on the current stream)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        step(options)
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(options)
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune(step, space: dict | None = None, start: dict | None = None, reps: int = 5, warmup: int = 2,
         sweeps: int = 2, cache_path: str | None = None, key: str | None = None):
    """Coordinate-descent search.  Returns (best options, best ms, log).

    With ``cache_path`` and ``key`` the result is read from / written to a JSON
    file, so a repeated run of the same workload skips the search.
    """
    space = dict(space or OPTION_SPACE)
    if cache_path and key and os.path.exists(cache_path):
        try:
            cached = json.load(open(cache_path)).get(key)
            if cached:
                return {int(k): v for k, v in cached["options"].items()}, cached["ms"], []
        except (OSError, ValueError):
            pass
    best = dict(DEFAULTS)
    best.update(start or {})
    best_ms = time_step(step, best, reps, warmup)
    log = [(dict(best), best_ms)]
    for _ in range(sweeps):
        improved = False
        for opt, values in space.items():
            for v in values:
                if best.get(opt) == v:
                    continue
                cand = dict(best)
                cand[opt] = v
                ms = time_step(step, cand, reps, warmup)
                log.append((cand, ms))
                if ms < best_ms * 0.995:
                    best, best_ms, improved = cand, ms, True
        if not improved:
            break
    if cache_path and key:
        data = {}
        if os.path.exists(cache_path):
            try:
                data = json.load(open(cache_path))
            except (OSError, ValueError):
                data = {}
        data[key] = {"options": {str(k): v for k, v in best.items()}, "ms": best_ms}
        with open(cache_path, "w") as fh:
            json.dump(data, fh, indent=1)
    return best, best_ms, log
