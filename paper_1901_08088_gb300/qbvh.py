"""Python surface of the qbvh library: the C entry points under the same names,
plus a small ``NeighborList`` owner class.

PyTorch provides device memory and streams only.  Inputs are CUDA tensors whose
data pointers go straight to the C ABI; outputs owned by the library are
exposed as non-owning tensor views (valid until the next build, query or
destroy on the same handle).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import QBVHError, check, lib

__all__ = [
    "QBVHError", "NeighborList",
    "qbvh_create", "qbvh_destroy", "qbvh_set_option", "qbvh_get_option",
    "qbvh_build", "qbvh_build_f64", "qbvh_build_batched", "qbvh_query", "qbvh_query_async", "qbvh_query_status",
    "qbvh_query_lj_async",
    "nlist_get", "qbvh_tree_get", "qbvh_lj_forward", "qbvh_lj_backward", "qbvh_pack_positions",
    "qbvh_lj_forward_noalloc", "qbvh_selftest_wait_timeout", "qbvh_strerror",
]


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


class _DevArray:
    """Minimal __cuda_array_interface__ holder for zero-copy tensor views."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {
            "shape": tuple(int(s) for s in shape), "typestr": typestr,
            "data": (int(ptr), False), "version": 3, "strides": None,
        }


def _view(ptr: int, shape, dtype: torch.dtype, device: int) -> torch.Tensor:
    if ptr == 0 or int(np.prod(shape)) == 0:
        return torch.empty(shape, dtype=dtype, device=f"cuda:{device}")
    typestr = {torch.int32: "<i4", torch.float32: "<f4", torch.float64: "<f8"}[dtype]
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device=f"cuda:{device}")


# ---------------------------------------------------------------- C entry points

def qbvh_strerror(code: int) -> str:
    return lib().qbvh_strerror(int(code)).decode()


def qbvh_create(device: int = 0) -> int:
    h = C.c_void_p()
    check(lib().qbvh_create(C.byref(h), int(device)), "qbvh_create")
    return h.value


def qbvh_destroy(h: int) -> None:
    check(lib().qbvh_destroy(h), "qbvh_destroy")


def qbvh_set_option(h: int, option: int, value: int) -> None:
    check(lib().qbvh_set_option(h, int(option), int(value)), "qbvh_set_option")


def qbvh_get_option(h: int, option: int) -> int:
    v = C.c_int()
    check(lib().qbvh_get_option(h, int(option), C.byref(v)), "qbvh_get_option")
    return v.value


def qbvh_build(h: int, pos4: torch.Tensor, L: float, n_types: int = 1, stream=None) -> int:
    """pos4: [n, 4] float32 CUDA tensor (x, y, z, type as int bits)."""
    n = int(pos4.shape[0])
    return lib().qbvh_build(h, _ptr(pos4) if n else None, n, float(np.float32(L)), int(n_types),
                            _stream_ptr(stream))


def qbvh_build_f64(h: int, pos4d: torch.Tensor, L: float, n_types: int = 1, stream=None) -> int:
    """pos4d: [n, 4] float64 CUDA tensor (x, y, z, type as a whole number); L in FP64."""
    n = int(pos4d.shape[0])
    return lib().qbvh_build_f64(h, _ptr(pos4d) if n else None, n, float(L), int(n_types), _stream_ptr(stream))


def qbvh_build_batched(h: int, pos4: torch.Tensor, offsets, Ls, n_types: int = 1, stream=None) -> int:
    off = np.ascontiguousarray(np.asarray(offsets, np.int32))
    Lh = np.ascontiguousarray(np.asarray(Ls, np.float32))
    n = int(pos4.shape[0])
    return lib().qbvh_build_batched(h, _ptr(pos4) if n else None, n, int(Lh.size),
                                    off.ctypes.data_as(C.c_void_p), Lh.ctypes.data_as(C.c_void_p),
                                    int(n_types), _stream_ptr(stream))


def _rl(r_list, n_types):
    r = np.asarray(r_list, np.float32)
    if r.ndim == 0:
        r = np.full((n_types, n_types), r, np.float32)
    return np.ascontiguousarray(r.reshape(n_types, n_types))


def qbvh_query(h: int, r_list, n_types: int, cap: int = 256, max_retries: int = 4, stream=None) -> int:
    r = _rl(r_list, n_types)
    return lib().qbvh_query(h, r.ctypes.data_as(C.c_void_p), int(cap), int(max_retries), _stream_ptr(stream))


def qbvh_query_async(h: int, r_list, n_types: int, cap: int, stream=None) -> int:
    r = _rl(r_list, n_types)
    return lib().qbvh_query_async(h, r.ctypes.data_as(C.c_void_p), int(cap), _stream_ptr(stream))


def qbvh_query_lj_async(h: int, pos4, r_list, n_types: int, cap: int, eps, sig, r_cut_host, e, U, F, dE, dS,
                        stream=None) -> int:
    """Traversal + LJ forward over the list it writes (fused where the library supports it)."""
    r = _rl(r_list, n_types)
    rc = np.ascontiguousarray(np.broadcast_to(np.asarray(r_cut_host, np.float32), (n_types, n_types)))
    return lib().qbvh_query_lj_async(h, _ptr(pos4), r.ctypes.data_as(C.c_void_p), int(cap), _ptr(eps), _ptr(sig),
                                     rc.ctypes.data_as(C.c_void_p), _ptr(e), _ptr(U), _ptr(F), _ptr(dE), _ptr(dS),
                                     _stream_ptr(stream))


def qbvh_query_status(h: int):
    m = C.c_int()
    rc = lib().qbvh_query_status(h, C.byref(m))
    return rc, m.value


def nlist_get(h: int):
    rows, counts = C.c_void_p(), C.c_void_p()
    cap, mx = C.c_int(), C.c_int()
    check(lib().nlist_get(h, C.byref(rows), C.byref(counts), C.byref(cap), C.byref(mx)), "nlist_get")
    return rows.value or 0, counts.value or 0, cap.value, mx.value


def qbvh_tree_get(h: int):
    nodes, leaves, order, seg_start, frames = (C.c_void_p() for _ in range(5))
    n_seg = C.c_int()
    check(lib().qbvh_tree_get(h, C.byref(nodes), C.byref(leaves), C.byref(order), C.byref(seg_start),
                              C.byref(frames), C.byref(n_seg)), "qbvh_tree_get")
    return (nodes.value or 0, leaves.value or 0, order.value or 0, seg_start.value or 0,
            frames.value or 0, n_seg.value)


def qbvh_lj_forward(h: int, pos4, eps, sig, r_cut_host, e, U, F, dE, dS, stream=None) -> int:
    rc = np.ascontiguousarray(np.asarray(r_cut_host, np.float32))
    return lib().qbvh_lj_forward(h, _ptr(pos4), _ptr(eps), _ptr(sig), rc.ctypes.data_as(C.c_void_p),
                                 _ptr(e), _ptr(U), _ptr(F), _ptr(dE), _ptr(dS), _stream_ptr(stream))


def qbvh_lj_backward(h: int, g, F, dE, dS, gpos, geps, gsig, stream=None) -> int:
    return lib().qbvh_lj_backward(h, _ptr(g), _ptr(F), _ptr(dE), _ptr(dS), _ptr(gpos), _ptr(geps),
                                  _ptr(gsig), _stream_ptr(stream))


def qbvh_lj_forward_noalloc(pos4, L, n_types, rows, counts, eps, sig, r_cut_host, e, U, F, dE, dS, status,
                            stream=None) -> int:
    """Allocation-free LJ pass over a caller-provided list (one system);
    `status` is a [1] int32 CUDA tensor that receives the device-side outcome."""
    rc = np.ascontiguousarray(np.asarray(r_cut_host, np.float32))
    n = int(pos4.shape[0])
    return lib().qbvh_lj_forward_noalloc(_ptr(pos4) if n else None, n, float(np.float32(L)), int(n_types),
                                         _ptr(rows) if n else None, _ptr(counts) if n else None,
                                         int(rows.shape[1]), _ptr(eps), _ptr(sig), rc.ctypes.data_as(C.c_void_p),
                                         _ptr(e), _ptr(U), _ptr(F), _ptr(dE), _ptr(dS), _ptr(status),
                                         _stream_ptr(stream))


def qbvh_selftest_wait_timeout(device: int = 0, stream=None) -> int:
    return lib().qbvh_selftest_wait_timeout(int(device), _stream_ptr(stream))


def qbvh_pack_positions(xyz: torch.Tensor, types, out4: torch.Tensor, stream=None) -> int:
    n = int(xyz.shape[0])
    return lib().qbvh_pack_positions(_ptr(xyz) if n else None, _ptr(types) if types is not None else None,
                                     n, _ptr(out4) if n else None, _stream_ptr(stream))


# ---------------------------------------------------------------- owner class

class NeighborList:
    """Owns one library handle: build the trees, query the list, read it back.

    >>> nl = NeighborList()
    >>> nl.build(pos4, L)                # pos4: [n, 4] float32 CUDA tensor
    >>> nl.query(3.4, cap=256)           # exact list within r_list = 3.4
    >>> rows, counts = nl.neighbors()    # non-owning views, [n, cap] and [n]
    """

    def __init__(self, device: int | None = None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        self.h = qbvh_create(self.device)
        self.n = 0
        self.n_types = 1
        self.n_sys = 1
        self.offsets = np.array([0, 0], np.int32)

    def close(self):
        if getattr(self, "h", None):
            qbvh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option: int, value: int):
        qbvh_set_option(self.h, option, value)

    def get_option(self, option: int) -> int:
        return qbvh_get_option(self.h, option)

    def build(self, pos4: torch.Tensor, L: float, n_types: int = 1, stream=None):
        check(qbvh_build(self.h, pos4, L, n_types, stream), "qbvh_build")
        self.n, self.n_types, self.n_sys = int(pos4.shape[0]), int(n_types), 1
        self.offsets = np.array([0, self.n], np.int32)
        return self

    def build_f64(self, pos4d: torch.Tensor, L: float, n_types: int = 1, stream=None):
        """Double-precision particle data (float64 [n, 4]); the list is exact in FP64."""
        check(qbvh_build_f64(self.h, pos4d, L, n_types, stream), "qbvh_build_f64")
        self.n, self.n_types, self.n_sys = int(pos4d.shape[0]), int(n_types), 1
        self.offsets = np.array([0, self.n], np.int32)
        return self

    def build_batched(self, pos4: torch.Tensor, offsets, Ls, n_types: int = 1, stream=None):
        check(qbvh_build_batched(self.h, pos4, offsets, Ls, n_types, stream), "qbvh_build_batched")
        self.n, self.n_types = int(pos4.shape[0]), int(n_types)
        self.offsets = np.asarray(offsets, np.int32)
        self.n_sys = int(self.offsets.size - 1)
        return self

    def query(self, r_list, cap: int = 256, max_retries: int = 4, stream=None, raise_on_error=True) -> int:
        rc = qbvh_query(self.h, r_list, self.n_types, cap, max_retries, stream)
        if raise_on_error:
            check(rc, "qbvh_query")
        return rc

    def query_async(self, r_list, cap: int, stream=None):
        check(qbvh_query_async(self.h, r_list, self.n_types, cap, stream), "qbvh_query_async")

    def query_lj_async(self, pos4, r_list, cap: int, eps, sig, r_cut, e=None, U=None, F=None, dE=None, dS=None,
                       stream=None):
        """Enqueue the traversal and the LJ energies/forces over its list; read
        the outcome with ``query_status`` after the stream completes."""
        check(qbvh_query_lj_async(self.h, pos4, r_list, self.n_types, cap, eps, sig, r_cut, e, U, F, dE, dS,
                                  stream), "qbvh_query_lj_async")

    def query_status(self):
        return qbvh_query_status(self.h)

    def neighbors(self):
        rows, counts, cap, _ = nlist_get(self.h)
        return (_view(rows, (self.n, cap), torch.int32, self.device),
                _view(counts, (self.n,), torch.int32, self.device))

    @property
    def cap(self) -> int:
        return nlist_get(self.h)[2]

    @property
    def max_count(self) -> int:
        return nlist_get(self.h)[3]

    def tree(self):
        nodes, leaves, order, seg_start, frames, n_seg = qbvh_tree_get(self.h)
        n = self.n
        return dict(
            nodes=_view(nodes, (n, 4), torch.int32, self.device),
            leaves=_view(leaves, (n, 4), torch.float32, self.device),
            order=_view(order, (n,), torch.int32, self.device),
            seg_start=_view(seg_start, (n_seg + 1,), torch.int32, self.device),
            frames=_view(frames, (n_seg, 8), torch.float32, self.device),
        )
