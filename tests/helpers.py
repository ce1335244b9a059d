"""Shared helpers for the GPU parity tests (inputs from workloads, references
from the oracle, results through the C ABI)."""
import numpy as np

import oracle
import workloads

BIG = np.iinfo(np.int32).max


def sorted_rows(rows, counts, cap=None):
    """Rows with entries past the count masked, each row sorted ascending."""
    rows = np.asarray(rows)
    cap = rows.shape[1] if cap is None else cap
    c = np.minimum(np.asarray(counts), cap)
    mask = np.arange(rows.shape[1])[None, :] < c[:, None]
    return np.sort(np.where(mask, rows, BIG), axis=1)


def assert_same_lists(rows_g, counts_g, rows_o, counts_o, idx=None):
    counts_g = np.asarray(counts_g)
    counts_o = np.asarray(counts_o)
    if idx is None:
        assert np.array_equal(counts_g, counts_o), np.nonzero(counts_g != counts_o)[0][:10]
        a = sorted_rows(rows_g, counts_g)
        b = sorted_rows(rows_o, counts_o)
        w = min(a.shape[1], b.shape[1])
        bad = np.nonzero((a[:, :w] != b[:, :w]).any(1))[0]
        assert bad.size == 0, bad[:10]
    else:
        assert np.array_equal(counts_g[idx], counts_o[idx])
        a = sorted_rows(rows_g[idx], counts_g[idx])
        b = sorted_rows(rows_o[idx], counts_o[idx])
        w = min(a.shape[1], b.shape[1])
        assert np.array_equal(a[:, :w], b[:, :w])


def gpu_list(system, cap=256, bundle=None, block=None, candidates=None, max_retries=4, traversal=None,
             node_format=None, method=None, grid_lanes=None, warp_particles=None, persistent=None):
    import torch
    from paper_1901_08088_gb300 import NeighborList, _lib

    nl = NeighborList(0)
    if bundle is not None:
        nl.set_option(_lib.QBVH_OPT_BUNDLE, bundle)
    if block is not None:
        nl.set_option(_lib.QBVH_OPT_QUERY_BLOCK, block)
    if candidates is not None:
        nl.set_option(_lib.QBVH_OPT_CANDIDATES, candidates)
    if traversal is not None:
        nl.set_option(_lib.QBVH_OPT_TRAVERSAL, traversal)
    if node_format is not None:
        nl.set_option(_lib.QBVH_OPT_NODE_FORMAT, node_format)
    if method is not None:
        nl.set_option(_lib.QBVH_OPT_METHOD, method)
    if warp_particles is not None:
        nl.set_option(_lib.QBVH_OPT_WARP_PARTICLES, warp_particles)
    if grid_lanes is not None:
        nl.set_option(_lib.QBVH_OPT_GRID_LANES, grid_lanes)
    if persistent is not None:
        nl.set_option(_lib.QBVH_OPT_PERSISTENT, persistent)
    pos4 = torch.from_numpy(workloads.pack_float4(system.pos, system.types)).cuda()
    nl.build(pos4, system.L, system.n_types)
    nl.query(system.r_list, cap=cap, max_retries=max_retries)
    rows, counts = nl.neighbors()
    return rows.cpu().numpy(), counts.cpu().numpy(), nl, pos4


def oracle_list(system, cap=256, method="cell"):
    return oracle.nlist(system.pos, system.L, system.r_list, system.types, system.n_types, cap=cap,
                        method=method)


def concat(systems):
    """Concatenate systems for a batched build: pos4, offsets, Ls."""
    pos4 = np.concatenate([workloads.pack_float4(s.pos, s.types) for s in systems])
    off = np.concatenate([[0], np.cumsum([s.n for s in systems])]).astype(np.int32)
    Ls = np.array([s.L for s in systems], np.float32)
    return pos4, off, Ls


def assert_same_lists_chunked(rows_dev, counts_g, rows_o, counts_o, chunk=1 << 17):
    """assert_same_lists over every row of a large list, read from the device
    view `rows_dev` ([n, cap] tensor) in chunks of rows so that the host never
    sorts the whole list at once."""
    counts_g = np.asarray(counts_g)
    counts_o = np.asarray(counts_o)
    bad = np.nonzero(counts_g != counts_o)[0]
    assert bad.size == 0, ("counts differ", bad[:10])
    n = counts_o.size
    w = int(min(max(int(counts_o.max(initial=0)), 1), rows_o.shape[1], rows_dev.shape[1]))
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        g = rows_dev[c0:c1, :w].cpu().numpy()
        a = sorted_rows(g, counts_g[c0:c1])
        b = sorted_rows(rows_o[c0:c1, :w], counts_o[c0:c1])
        bad = np.nonzero((a != b).any(1))[0]
        assert bad.size == 0, ("rows differ", (c0 + bad[:10]).tolist())
