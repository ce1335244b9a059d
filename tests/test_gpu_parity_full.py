"""Full-size parity of the headline configurations, every row.

* The N = 2,097,152 fluid (the benchmark's workload): every one of the 2M
  rows against the oracle's cell list, under the options the benchmark's
  autotuner picks (K = 64, 128-thread blocks, 10-bit quantized nodes; earlier
  K = 32 with FP32 nodes), under every node format, with two and four lanes
  per particle, and under the one-thread-per-particle walk of Alg. 1 as
  written; plus the FP64 band check of the FP32 decision on a sample.
* The differentiable two-type workload (32 systems x 65,536 particles, one
  batched build): every row of every system against the oracle of that
  system alone, with one tree per type (the paper's layout, Sec. 1 and 5) and
  with one tree per system (the layout the benchmark uses when every type
  pair shares a radius).

Rows are compared as sorted sets (row order is unspecified), bit for bit.
"""
import numpy as np
import pytest

import oracle
import workloads
from helpers import assert_same_lists_chunked, concat

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CAP = 256


@pytest.fixture(scope="module")
def fluid_2m():
    s = workloads.workload("lj_n2097152_rho0.8", seed=0)
    ro, co = oracle.nlist(s.pos, s.L, s.r_list, cap=CAP)
    return s, ro, co


@pytest.mark.parametrize("opts", [
    dict(bundle=32, block=256, node_format=1, traversal=1, warp_particles=32),   # the benchmark's choice
    dict(bundle=32, block=256, node_format=0, traversal=1, warp_particles=32),   # 10-bit quantized nodes
    dict(bundle=16, block=128, node_format=0, traversal=0, warp_particles=32),   # Alg. 1 one thread per particle
    dict(bundle=16, block=128, node_format=1, traversal=1, warp_particles=16),   # two lanes per particle
    dict(bundle=64, block=256, node_format=0, traversal=1, warp_particles=32),   # 64-leaf bundles
    dict(bundle=64, block=256, node_format=2, traversal=1, warp_particles=32),   # 21-bit nodes
    dict(bundle=64, block=128, node_format=0, traversal=1, warp_particles=32),   # the benchmark's current choice
    dict(bundle=64, block=128, node_format=1, traversal=1, warp_particles=32),   # FP32 nodes, 64-leaf bundles
    dict(bundle=64, block=128, node_format=0, traversal=1, warp_particles=8),    # four lanes per particle, filtered
], ids=["bench_fp32_nodes", "quantized_nodes", "thread_per_particle", "two_lanes_per_particle", "bundles_64",
        "nodes_21bit", "bench_current", "fp32_nodes_64", "four_lanes_per_particle"])
def test_all_2m_rows_equal_cell_list(fluid_2m, opts):
    import torch

    from paper_1901_08088_gb300 import NeighborList, _lib

    s, ro, co = fluid_2m
    nl = NeighborList(0)
    nl.set_option(_lib.QBVH_OPT_BUNDLE, opts["bundle"])
    nl.set_option(_lib.QBVH_OPT_QUERY_BLOCK, opts["block"])
    nl.set_option(_lib.QBVH_OPT_NODE_FORMAT, opts["node_format"])
    nl.set_option(_lib.QBVH_OPT_TRAVERSAL, opts["traversal"])
    nl.set_option(_lib.QBVH_OPT_WARP_PARTICLES, opts["warp_particles"])
    pos4 = torch.from_numpy(workloads.pack_float4(s.pos, s.types)).cuda()
    nl.build(pos4, s.L)
    nl.query(s.r_list, cap=CAP)
    rows, counts = nl.neighbors()
    cg = counts.cpu().numpy()
    assert_same_lists_chunked(rows, cg, ro, co)
    assert nl.max_count == int(co.max())
    idx = np.sort(np.random.default_rng(3).choice(s.n, 4096, replace=False))
    rg = rows[torch.from_numpy(idx).cuda()].cpu().numpy()
    full = np.zeros((s.n, rg.shape[1]), np.int32)
    full[idx] = rg
    nbad, bad = oracle.band_check(s.pos, s.L, s.r_list, full, cg, sample=idx)
    assert nbad == 0, bad
    nl.close()


@pytest.mark.parametrize("type_trees", [1, 0], ids=["tree_per_type", "tree_per_system"])
def test_config5_every_row_of_every_system(type_trees):
    import torch

    from paper_1901_08088_gb300 import NeighborList, _lib

    systems = workloads.workload("lj2type_32x65536", seed=0)
    pos4, off, Ls = concat(systems)
    nl = NeighborList(0)
    nl.set_option(_lib.QBVH_OPT_TYPE_TREES, type_trees)
    nl.build_batched(torch.from_numpy(pos4).cuda(), off, Ls, n_types=2)
    nl.query(systems[0].r_list, cap=CAP)
    rows, counts = nl.neighbors()
    cg = counts.cpu().numpy()
    for k, q in enumerate(systems):
        a, b = int(off[k]), int(off[k + 1])
        ro, co = oracle.nlist(q.pos, q.L, q.r_list, q.types, q.n_types, cap=CAP)
        # the batched list holds concatenated indices: shift the oracle's
        ro = np.where(np.arange(CAP)[None, :] < co[:, None], ro + a, ro)
        assert_same_lists_chunked(rows[a:b], cg[a:b], ro, co)
    nl.close()
