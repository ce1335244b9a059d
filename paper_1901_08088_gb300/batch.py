"""Many independent periodic systems through one launch sequence.

``BatchedNeighborList`` builds the trees of every system (one per system and
type) and their neighbor lists with the library's batched build
(``qbvh_build_batched``) and one traversal launch, captured once into a CUDA
graph and replayed every step.  The graph ends with the 16-byte status copy;
after a replay the host reads it and, if some row outgrew the capacity, raises
the capacity and captures again (the tree is rebuilt inside the graph, so a
replay always reflects the current positions in the input buffer).

``PerSystemLoop`` is the comparison point: the same kernels, one system at a
time (one handle per system, all launches on one stream, one wait at the end).
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib
from .qbvh import NeighborList, check

__all__ = ["BatchedNeighborList", "PerSystemLoop"]


class BatchedNeighborList:
    """Batched build + query of ``n_sys`` systems replayed from a CUDA graph.

    pos4    : [N_total, 4] float32 CUDA tensor (the graph reads this buffer;
              update it in place between replays)
    offsets : [n_sys + 1] system offsets into pos4
    Ls      : [n_sys] cubic box edges
    """

    def __init__(self, pos4: torch.Tensor, offsets, Ls, r_list, n_types: int = 1, cap: int = 128,
                 options: dict | None = None, device: int | None = None, max_regrow: int = 4):
        self.nl = NeighborList(device)
        for k, v in (options or {}).items():
            self.nl.set_option(k, v)
        self.pos4 = pos4
        self.offsets = np.asarray(offsets, np.int32)
        self.Ls = np.asarray(Ls, np.float32)
        self.n_types = int(n_types)
        self.r_list = r_list
        self.cap = int(cap)
        self.max_regrow = int(max_regrow)
        self.graph = None
        self.captures = 0

    def _enqueue(self):
        self.nl.build_batched(self.pos4, self.offsets, self.Ls, self.n_types)
        self.nl.query_async(self.r_list, self.cap)

    def capture(self):
        """Warm up at the current sizes (allocations happen here), then capture."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._enqueue()
        side.synchronize()
        rc, mx = self.nl.query_status()
        if rc == _lib.QBVH_ERR_OVERFLOW:
            self.cap = int((mx + 31) // 32 * 32)
            with torch.cuda.stream(side):
                self._enqueue()
            side.synchronize()
            rc, mx = self.nl.query_status()
        check(rc, "batched warm-up")
        torch.cuda.current_stream().wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._enqueue()
        self.captures += 1
        return self

    def replay(self):
        """Enqueue one build + query on the current stream (no host wait)."""
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def enqueue_eager(self):
        """The same build + query launched directly instead of from the graph
        (no host wait); read the outcome with ``status`` after the stream has run."""
        self._enqueue()

    def status(self) -> int:
        """After the stream has finished a replay: QBVH_OK, or grows cap and recaptures on overflow."""
        rc, mx = self.nl.query_status()
        regrow = 0
        while rc == _lib.QBVH_ERR_OVERFLOW and regrow < self.max_regrow:
            self.cap = int((mx + 31) // 32 * 32)
            self.capture()
            self.graph.replay()
            torch.cuda.current_stream().synchronize()
            rc, mx = self.nl.query_status()
            regrow += 1
        return rc

    def run(self) -> int:
        """One step: replay, wait, check."""
        self.replay()
        torch.cuda.current_stream().synchronize()
        return self.status()

    def neighbors(self):
        return self.nl.neighbors()

    def close(self):
        self.graph = None
        self.nl.close()


class PerSystemLoop:
    """The same build + query, one system at a time, each with its own handle."""

    def __init__(self, pos4: torch.Tensor, offsets, Ls, r_list, n_types: int = 1, cap: int = 128,
                 options: dict | None = None, device: int | None = None):
        self.offsets = np.asarray(offsets, np.int32)
        self.Ls = np.asarray(Ls, np.float32)
        self.views = [pos4[self.offsets[k]:self.offsets[k + 1]] for k in range(len(self.Ls))]
        self.handles = []
        for _ in range(len(self.Ls)):
            nl = NeighborList(device)
            for k, v in (options or {}).items():
                nl.set_option(k, v)
            self.handles.append(nl)
        self.r_list = r_list
        self.n_types = int(n_types)
        self.cap = int(cap)

    def enqueue(self):
        for nl, p, L in zip(self.handles, self.views, self.Ls):
            nl.build(p, float(L), self.n_types)
            nl.query_async(self.r_list, self.cap)

    def run(self) -> int:
        self.enqueue()
        torch.cuda.current_stream().synchronize()
        worst = _lib.QBVH_OK
        for nl in self.handles:
            rc, _ = nl.query_status()
            if rc != _lib.QBVH_OK:
                worst = rc
        return worst

    def close(self):
        for nl in self.handles:
            nl.close()
