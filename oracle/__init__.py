"""CPU oracle for the quantized-BVH neighbor search -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The product library
(``paper_1901_08088_gb300``) never imports, links or runs it, and this package
imports nothing from the product.

Contents (C sources compiled with gcc into ``_oracle.so``):

* ``nlist_ref.c`` -- the neighbor-list definition (Sec. 1 / Sec. 4): O(N^2)
  brute force, a 27-cell uniform-grid list (Sec. 1, Fig. 1b) with the same
  FP32 decision expression, and an FP64 band check.
* ``lbvh_ref.c``  -- the quantized LBVH built step by step (Sec. 2.1, 2.2,
  Fig. 3): Morton binning, stable sort, recursive hierarchy, fit, ropes,
  outward quantization with IEEE directed rounding (Sec. 3).
* ``lj_ref.c``    -- FP64 truncated-shifted Lennard-Jones energy (Eq. 1),
  forces and per-type-pair parameter gradients.
* ``nlist64_ref.c`` -- neighbor lists of double-precision particle data
  (Sec. 2.2): brute force and 27-cell list with one pinned FP64 decision
  expression.
* ``cand_ref.c``  -- candidate lists of Alg. 1 without the exact leaf filter
  (Sec. 2.3): every leaf whose box (10-bit or 21-bit quantized, or the FP32
  point) the padded sphere overlaps, under every periodic image whose sphere
  overlaps the tree's root box; brute force.

Pins: every function here is checked by ``tests/test_oracle_*.py`` against
closed forms, brute force, golden hand-derived fixtures and invariants.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")
_SRCS = ["nlist_ref.c", "lbvh_ref.c", "lj_ref.c", "nlist64_ref.c", "cand_ref.c"]
_lock = threading.Lock()
_lib = None

END = np.int32(-(2 ** 31))

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
          "-frounding-math", "-fno-fast-math", "-fsigned-char"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (idempotent)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    if not force and os.path.exists(_SO):
        so_m = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_m for s in srcs):
            return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            P = C.c_void_p
            i32, f32, f64 = C.c_int, C.c_float, C.c_double
            L.or_nlist_brute.argtypes = [i32, P, P, f32, i32, P, i32, P, P]
            L.or_nlist_brute.restype = i32
            L.or_nlist_cell.argtypes = [i32, P, P, f32, i32, P, i32, P, P]
            L.or_nlist_cell.restype = i32
            L.or_band_check.argtypes = [i32, P, P, f32, i32, P, f64, i32, P, P, i32, P, i32, P]
            L.or_band_check.restype = C.c_long
            L.or_nlist64_brute.argtypes = [i32, P, P, f64, i32, P, i32, P, P]
            L.or_nlist64_brute.restype = i32
            L.or_nlist64_cell.argtypes = [i32, P, P, f64, i32, P, i32, P, P]
            L.or_nlist64_cell.restype = i32
            L.or_num_threads.argtypes = []
            L.or_num_threads.restype = i32
            L.or_morton.argtypes = [i32, P, P, P, P]
            L.or_morton.restype = None
            L.or_lbvh_build.argtypes = [i32, P, P, i32, P, i32, P, P, P, P, P, P, P]
            L.or_lbvh_build.restype = i32
            L.or_lbvh_topology.argtypes = [i32, P, P, i32, P, P, P, P, P, P, P, P, P]
            L.or_lbvh_topology.restype = i32
            L.or_quantize_box.argtypes = [P, P, P, P, P, P]
            L.or_quantize_box.restype = None
            L.or_dequantize.argtypes = [P, P, P, P, P, P]
            L.or_dequantize.restype = None
            L.or_quantize_box_q.argtypes = [P, P, P, P, C.c_long, P, P]
            L.or_quantize_box_q.restype = None
            L.or_frame_width.argtypes = [P, P, C.c_long, P]
            L.or_frame_width.restype = None
            L.or_lj_fp64.argtypes = [i32, P, P, P, f32, i32, P, P, P, i32, P, P, P, P, P, P, P]
            L.or_lj_fp64.restype = i32
            L.or_candidates.argtypes = [i32, P, P, f32, i32, P, P, P, i32, i32, P, P]
            L.or_candidates.restype = i32
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def num_threads() -> int:
    return int(lib().or_num_threads())


# ---------------------------------------------------------------- neighbor lists

def _rl_matrix(r_list, nt):
    rl = np.asarray(r_list, np.float32)
    if rl.ndim == 0:
        rl = np.full((nt, nt), rl, np.float32)
    return _c(rl.reshape(nt, nt), np.float32)


def nlist(pos, L, r_list, types=None, n_types=1, cap=256, method="cell"):
    """Exact neighbor list. Returns (rows [n,cap] int32 sorted asc, counts [n] int32)."""
    pos = _c(pos, np.float32).reshape(-1, 3)
    n = pos.shape[0]
    types = np.zeros(n, np.int32) if types is None else _c(types, np.int32)
    rl = _rl_matrix(r_list, n_types)
    rows = np.full((n, cap), -1, np.int32)
    counts = np.zeros(n, np.int32)
    fn = lib().or_nlist_brute if method == "brute" else lib().or_nlist_cell
    rc = fn(n, _p(pos), _p(types), float(np.float32(L)), n_types, _p(rl), cap, _p(rows), _p(counts))
    if rc != 0:
        raise RuntimeError(f"oracle nlist failed ({rc})")
    return rows, counts


def candidates(pos, L, r_list, types=None, n_types=1, cap=256, leaf_bits=10):
    """Candidate lists of Alg. 1 (no exact leaf filter, one tree per type),
    against leaf boxes quantized to 10 or 21 bits, or the FP32 points
    (leaf_bits=0).  Returns (rows [n,cap] int32 sorted asc, counts [n] int32);
    an index appears once per periodic image that lists it."""
    pos = _c(pos, np.float32).reshape(-1, 3)
    n = pos.shape[0]
    types = np.zeros(n, np.int32) if types is None else _c(types, np.int32)
    rl = _rl_matrix(r_list, n_types)
    L32 = np.float32(L)
    tree = lbvh_build(pos, types, np.full(n_types, L32, np.float32))
    rows = np.full((n, cap), -1, np.int32)
    counts = np.zeros(n, np.int32)
    rc = lib().or_candidates(n, _p(pos), _p(types), float(L32), n_types, _p(rl), _p(tree["root"]),
                             _p(tree["frame"]), int(leaf_bits), cap, _p(rows), _p(counts))
    if rc != 0:
        raise RuntimeError(f"oracle candidates failed ({rc})")
    return rows, counts


def nlist64(pos, L, r_list, types=None, n_types=1, cap=256, method="cell"):
    """Exact neighbor list of FP64 positions (FP64 decision, FP32 list radii).
    Returns (rows [n,cap] int32 sorted asc, counts [n] int32)."""
    pos = _c(pos, np.float64).reshape(-1, 3)
    n = pos.shape[0]
    types = np.zeros(n, np.int32) if types is None else _c(types, np.int32)
    rl = _rl_matrix(r_list, n_types)
    rows = np.full((n, cap), -1, np.int32)
    counts = np.zeros(n, np.int32)
    fn = lib().or_nlist64_brute if method == "brute" else lib().or_nlist64_cell
    rc = fn(n, _p(pos), _p(types), float(L), n_types, _p(rl), cap, _p(rows), _p(counts))
    if rc != 0:
        raise RuntimeError(f"oracle nlist64 failed ({rc})")
    return rows, counts


def band_check(pos, L, r_list, rows, counts, types=None, n_types=1, band=1e-6,
               sample=None, max_bad=16):
    """FP64 check of an FP32 list; returns (violations, [(i, j), ...])."""
    pos = _c(pos, np.float32).reshape(-1, 3)
    n = pos.shape[0]
    types = np.zeros(n, np.int32) if types is None else _c(types, np.int32)
    rl = _rl_matrix(r_list, n_types)
    rows = _c(rows, np.int32)
    counts = _c(counts, np.int32)
    cap = rows.shape[1]
    smp = None if sample is None else _c(sample, np.int32)
    bad = np.zeros(2 * max_bad, np.int32)
    nbad = lib().or_band_check(n, _p(pos), _p(types), float(np.float32(L)), n_types, _p(rl),
                               float(band), cap, _p(rows), _p(counts),
                               0 if smp is None else smp.size, _p(smp), max_bad, _p(bad))
    k = min(int(nbad), max_bad)
    return int(nbad), [(int(bad[2 * t]), int(bad[2 * t + 1])) for t in range(k)]


def rows_as_sets(rows, counts):
    cap = rows.shape[1]
    return [frozenset(rows[i, : min(int(counts[i]), cap)].tolist()) for i in range(rows.shape[0])]


# ---------------------------------------------------------------- LBVH

def morton(pos, L, seg=None, Lseg=None):
    pos = _c(pos, np.float32).reshape(-1, 3)
    n = pos.shape[0]
    seg = np.zeros(n, np.int32) if seg is None else _c(seg, np.int32)
    Lseg = _c(np.atleast_1d(np.float32(L) if Lseg is None else Lseg), np.float32)
    out = np.zeros(n, np.uint32)
    lib().or_morton(n, _p(pos), _p(seg), _p(Lseg), _p(out))
    return out


def lbvh_build(pos, seg, Lseg, bundle_k=1):
    """Quantized LBVH of every segment. Returns a dict of numpy arrays."""
    pos = _c(pos, np.float32).reshape(-1, 3)
    n = pos.shape[0]
    seg = _c(seg, np.int32)
    Lseg = _c(np.atleast_1d(Lseg), np.float32)
    ns = Lseg.size
    out = dict(
        codes=np.zeros(n, np.uint32), order=np.zeros(n, np.int32),
        seg_start=np.zeros(ns + 1, np.int32), nodes=np.zeros((n, 4), np.int32),
        leaves=np.zeros((n, 4), np.float32), root=np.zeros((ns, 6), np.float32),
        frame=np.zeros((ns, 6), np.float32))
    rc = lib().or_lbvh_build(n, _p(pos), _p(seg), ns, _p(Lseg), int(bundle_k),
                             _p(out["codes"]), _p(out["order"]), _p(out["seg_start"]),
                             _p(out["nodes"]), _p(out["leaves"]), _p(out["root"]),
                             _p(out["frame"]))
    if rc != 0:
        raise RuntimeError("oracle lbvh_build rejected its input")
    return out


def lbvh_topology(pos, seg, Lseg):
    pos = _c(pos, np.float32).reshape(-1, 3)
    n = pos.shape[0]
    seg = _c(seg, np.int32)
    Lseg = _c(np.atleast_1d(Lseg), np.float32)
    ns = Lseg.size
    t = {k: np.zeros(n, np.int32) for k in
         ("left", "right", "first", "last", "rope_int", "rope_leaf", "order")}
    t["seg_start"] = np.zeros(ns + 1, np.int32)
    rc = lib().or_lbvh_topology(n, _p(pos), _p(seg), ns, _p(Lseg), _p(t["left"]), _p(t["right"]),
                                _p(t["first"]), _p(t["last"]), _p(t["rope_int"]),
                                _p(t["rope_leaf"]), _p(t["order"]), _p(t["seg_start"]))
    if rc != 0:
        raise RuntimeError("oracle lbvh_topology rejected its input")
    return t


def quantize_box(lo, hi, R_lo, h, bits=10):
    """Outward quantization of a box onto the bin edges 0..2^bits - 1."""
    a = [_c(v, np.float32) for v in (lo, hi, R_lo, h)]
    qlo = np.zeros(3, np.uint32)
    qhi = np.zeros(3, np.uint32)
    if bits == 10:
        lib().or_quantize_box(*[_p(v) for v in a], _p(qlo), _p(qhi))
    else:
        lib().or_quantize_box_q(*[_p(v) for v in a], (1 << bits) - 1, _p(qlo), _p(qhi))
    return qlo, qhi


def frame_width(R_lo, R_hi, bits):
    """Bin width per axis of a root box with 2^bits - 1 bins (rounded up)."""
    h = np.zeros(3, np.float32)
    lib().or_frame_width(_p(_c(R_lo, np.float32)), _p(_c(R_hi, np.float32)), (1 << bits) - 1, _p(h))
    return h


def dequantize(qlo, qhi, R_lo, h):
    a = [_c(qlo, np.uint32), _c(qhi, np.uint32), _c(R_lo, np.float32), _c(h, np.float32)]
    lo = np.zeros(3, np.float32)
    hi = np.zeros(3, np.float32)
    lib().or_dequantize(*[_p(v) for v in a], _p(lo), _p(hi))
    return lo, hi


def unpack10(word):
    """Packed qx<<20 | qy<<10 | qz (bits 30-31 ignored) -> (qx, qy, qz)."""
    w = np.asarray(word).astype(np.int64) & 0x3FFFFFFF
    return np.stack([(w >> 20) & 1023, (w >> 10) & 1023, w & 1023], axis=-1)


# ---------------------------------------------------------------- Lennard-Jones

def lj_fp64(pos32, types, L, eps, sig, r_cut, rows, counts, pos64=None, n_types=None):
    """FP64 energy, per-particle energy, forces and dU/deps, dU/dsig."""
    pos32 = _c(pos32, np.float32).reshape(-1, 3)
    n = pos32.shape[0]
    nt = int(n_types if n_types is not None else np.asarray(eps).reshape(-1).size ** 0.5 + 0.5)
    pos64 = pos32.astype(np.float64) if pos64 is None else _c(pos64, np.float64).reshape(-1, 3)
    types = _c(types, np.int32)
    eps = _c(np.asarray(eps, np.float64).reshape(nt, nt), np.float64)
    sig = _c(np.asarray(sig, np.float64).reshape(nt, nt), np.float64)
    rc = _c(np.broadcast_to(np.asarray(r_cut, np.float32), (nt, nt)), np.float32)
    rows = _c(rows, np.int32)
    counts = _c(counts, np.int32)
    U = np.zeros(1, np.float64)
    e = np.zeros(n, np.float64)
    F = np.zeros((n, 3), np.float64)
    dE = np.zeros((nt, nt), np.float64)
    dS = np.zeros((nt, nt), np.float64)
    r = lib().or_lj_fp64(n, _p(pos32), _p(pos64), _p(types), float(np.float32(L)), nt, _p(eps),
                         _p(sig), _p(rc), rows.shape[1], _p(rows), _p(counts), _p(U), _p(e),
                         _p(F), _p(dE), _p(dS))
    if r != 0:
        raise RuntimeError("oracle lj rejected its input")
    return dict(U=float(U[0]), e=e, F=F, dE=dE, dS=dS)
