"""The traversal with its packet queue (QBVH_OPT_PERSISTENT = 1): resident
warps take packets of 32 Z-order particles from a device counter instead of
one packet per warp of the grid.  Which warp walks a packet must not change
the list: checked bit for bit against the oracle through the C ABI for one
type under the three node formats, ragged sizes, several types with per-pair
radii (packets taken from the end of the sorted order, sparse trees in the
leading blocks), a batched ensemble (64-bit keys), repeated queries, a CUDA
graph replay and every row of the N = 2M bench fluid.
"""
import numpy as np
import pytest

import workloads
from helpers import assert_same_lists, assert_same_lists_chunked, concat, gpu_list, oracle_list

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("node_format", [0, 1, 2])
@pytest.mark.parametrize("bundle,block", [(16, 128), (64, 256), (64, 64)])
def test_queue_config1_equals_bruteforce(node_format, bundle, block):
    s = workloads.workload("lj_n4096_rho0.6", seed=21)
    rg, cg, nl, _ = gpu_list(s, node_format=node_format, bundle=bundle, block=block, persistent=1)
    ro, co = oracle_list(s, method="brute")
    assert_same_lists(rg, cg, ro, co)
    assert nl.max_count == int(co.max())
    nl.close()


@pytest.mark.parametrize("n", [1, 2, 31, 33, 1000, 12345, 70001])
def test_queue_ragged_sizes(n):
    rng = np.random.default_rng(n)
    L = np.float32(max(8.0, (n / 0.5) ** (1 / 3)))
    pos = rng.uniform(0, L, size=(n, 3)).astype(np.float32)
    pos[pos >= L] = 0
    rl = np.full((1, 1), 2.5, np.float32)
    s = workloads.System(pos=pos, types=np.zeros(n, np.int32), L=L, n_types=1, r_list=rl, r_cut=rl.copy())
    rg, cg, nl, _ = gpu_list(s, persistent=1)
    ro, co = oracle_list(s, method="brute" if n < 20000 else "cell")
    assert_same_lists(rg, cg, ro, co)
    nl.close()


def test_queue_several_types_and_sparse_trees():
    rng = np.random.default_rng(23)
    L = np.float32(60.0)
    counts = [60000, 3000, 1, 0]
    types = np.repeat(np.arange(4, dtype=np.int32), counts)
    types = types[rng.permutation(types.size)]
    pos = rng.uniform(0, L, size=(types.size, 3)).astype(np.float32)
    pos[pos >= L] = 0
    rl = np.array([[2.5, 4.0, 3.0, 2.0], [4.0, 6.0, 5.0, 2.0], [3.0, 5.0, 7.0, 2.0], [2.0, 2.0, 2.0, 2.0]],
                  np.float32)
    s = workloads.System(pos=pos, types=types, L=L, n_types=4, r_list=rl, r_cut=rl.copy())
    rg, cg, nl, _ = gpu_list(s, persistent=1)
    ro, co = oracle_list(s)
    assert_same_lists(rg, cg, ro, co)
    nl.close()
    m = workloads.binary_mixture(seed=3, L=40.0, n_large=20, n_small=25000)
    rg, cg, nl, _ = gpu_list(m, cap=512, persistent=1)
    ro, co = oracle_list(m, cap=512)
    assert_same_lists(rg, cg, ro, co)
    nl.close()


def test_queue_batched_ensemble_and_repeats():
    import torch

    from paper_1901_08088_gb300 import NeighborList, _lib

    systems = workloads.batched_ensemble(seed=7, n_sys=24, n_min=250, n_max=6000)
    pos4, off, Ls = concat(systems)
    nl = NeighborList(0)
    nl.set_option(_lib.QBVH_OPT_PERSISTENT, 1)
    nl.build_batched(torch.from_numpy(pos4).cuda(), off, Ls)
    first = None
    for _ in range(3):
        nl.query(systems[0].r_list)
        rows, counts = nl.neighbors()
        rows, counts = rows.cpu().numpy(), counts.cpu().numpy()
        if first is None:
            first = (rows.copy(), counts.copy())
        else:
            # the same entries in the same order: a packet's walk does not
            # depend on which warp takes it
            mask = np.arange(rows.shape[1])[None, :] < counts[:, None]
            assert np.array_equal(counts, first[1])
            assert np.array_equal(np.where(mask, rows, -1), np.where(mask, first[0], -1))
    for k, s in enumerate(systems):
        a, b = off[k], off[k + 1]
        ro, co = oracle_list(s, method="brute" if s.n < 3000 else "cell")
        assert_same_lists(rows[a:b] - a, counts[a:b], ro, co)
    nl.close()


def test_queue_graph_replay():
    """The queue counter is reset by the query's own memset, so a captured
    build + query replays correctly."""
    import torch

    from paper_1901_08088_gb300 import NeighborList, _lib

    s = workloads.workload("lj_n4096_rho0.6", seed=24)
    pos4 = torch.from_numpy(workloads.pack_float4(s.pos, s.types)).cuda()
    nl = NeighborList(0)
    nl.set_option(_lib.QBVH_OPT_PERSISTENT, 1)
    nl.build(pos4, s.L)
    nl.query(s.r_list)   # sizes the buffers before capture
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        nl.build(pos4, s.L, stream=stream)
        nl.query_async(s.r_list, 256, stream=stream)
    ro, co = oracle_list(s, method="brute")
    for _ in range(3):
        g.replay()
        torch.cuda.synchronize()
        rc, mx = nl.query_status()
        assert rc == 0 and mx == int(co.max())
        rows, counts = nl.neighbors()
        assert_same_lists(rows.cpu().numpy(), counts.cpu().numpy(), ro, co)
    nl.close()


@pytest.mark.slow
def test_queue_all_2m_rows():
    s = workloads.workload("lj_n2097152_rho0.8", seed=0)
    _, cg, nl, _ = gpu_list(s, bundle=64, block=128, node_format=0, persistent=1)
    ro, co = oracle_list(s)
    rows_dev, _ = nl.neighbors()
    assert_same_lists_chunked(rows_dev, cg, ro, co)
    nl.close()
