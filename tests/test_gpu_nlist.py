"""GPU parity: the CUDA build + traversal against the CPU oracle, through the C ABI.

Neighbor sets are compared bit-exactly (row order is unspecified, so rows are
compared as sorted sets); tree words (Morton order, leaves, quantized nodes,
frames) are compared bit-exactly with the oracle's step-by-step construction.
"""
import numpy as np
import pytest

import oracle
import workloads
from helpers import assert_same_lists, gpu_list, oracle_list

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg1():
    return workloads.workload("lj_n4096_rho0.6", seed=0)


@pytest.mark.parametrize("node_format", [0, 1, 2])
@pytest.mark.parametrize("traversal,wp", [(0, 32), (1, 32), (1, 16), (1, 8), (1, 4), (1, 2), (1, 1)])
@pytest.mark.parametrize("bundle,block", [(1, 128), (4, 128), (8, 64), (2, 256), (16, 128), (32, 32)])
def test_config1_exact_list_equals_bruteforce(cfg1, bundle, block, traversal, node_format, wp):
    rg, cg, nl, _ = gpu_list(cfg1, bundle=bundle, block=block, traversal=traversal, node_format=node_format,
                             warp_particles=wp)
    ro, co = oracle_list(cfg1, method="brute")
    assert_same_lists(rg, cg, ro, co)
    assert nl.max_count == co.max()
    nl.close()


@pytest.mark.parametrize("node_format", [0, 1, 2])
@pytest.mark.parametrize("n", [4096, 12345, 33, 65, 1000])
@pytest.mark.parametrize("bundle", [33, 48, 64])
def test_bundles_wider_than_a_warp(bundle, n, node_format):
    # bundles of more than 32 leaves are filtered 32 leaves at a time
    L = max(8.0, (n / 0.6) ** (1 / 3))
    s = _uniform(n, L, 2.5, seed=n + bundle)
    rg, cg, nl, _ = gpu_list(s, bundle=bundle, node_format=node_format, block=256)
    ro, co = oracle_list(s, method="brute")
    assert_same_lists(rg, cg, ro, co)
    nl.close()


@pytest.mark.parametrize("bundle", [1, 4, 64])
def test_tree_words_equal_oracle(cfg1, bundle):
    import torch

    _, _, nl, _ = gpu_list(cfg1, bundle=bundle)
    t = {k: v.cpu() for k, v in nl.tree().items()}
    o = oracle.lbvh_build(cfg1.pos, cfg1.types, [cfg1.L], bundle_k=bundle)
    assert np.array_equal(t["order"].numpy(), o["order"])
    assert np.array_equal(t["seg_start"].numpy(), o["seg_start"])
    assert np.array_equal(t["leaves"].view(torch.int32).numpy(), o["leaves"].view(np.int32))
    n = cfg1.n
    assert np.array_equal(t["nodes"].numpy()[: n - 1], o["nodes"][: n - 1])
    assert np.array_equal(t["frames"].numpy()[:, :6].view(np.int32), o["frame"].view(np.int32))
    nl.close()


def _uniform(n, L, r, seed, n_types=1):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, L, size=(n, 3)).astype(np.float32)
    pos[pos >= np.float32(L)] = 0
    types = rng.integers(0, n_types, n).astype(np.int32)
    rl = np.full((n_types, n_types), r, np.float32)
    return workloads.System(pos=pos, types=types, L=np.float32(L), n_types=n_types, r_list=rl,
                            r_cut=rl.copy())


@pytest.mark.parametrize("traversal,node_format,wp", [(0, 0, 32), (1, 0, 32), (1, 1, 32), (1, 0, 16), (1, 1, 8),
                                                     (1, 1, 4), (1, 0, 2), (1, 1, 1), (1, 2, 32), (0, 2, 32),
                                                     (1, 2, 4)])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 33, 255, 4095, 4097, 12345])
def test_ragged_sizes(n, traversal, node_format, wp):
    L = max(8.0, (n / 0.5) ** (1 / 3))
    s = _uniform(n, L, 2.5, seed=n)
    rg, cg, nl, _ = gpu_list(s, traversal=traversal, node_format=node_format, warp_particles=wp)
    ro, co = oracle_list(s, method="brute")
    assert_same_lists(rg, cg, ro, co)
    nl.close()


def test_coincident_and_identical_particles():
    s = _uniform(600, 10.0, 2.0, seed=1)
    s.pos[100:200] = s.pos[100]        # 100 coincident particles
    s.pos[300:310] = np.float32(0.0)   # particles exactly at the box corner
    rg, cg, nl, _ = gpu_list(s)
    ro, co = oracle_list(s, cap=256, method="brute")
    assert_same_lists(rg, cg, ro, co)
    nl.close()
    # every particle at one point: degenerate root box (zero-width bins)
    same = _uniform(50, 10.0, 2.0, seed=2)
    same.pos[:] = np.float32(3.25)
    rg, cg, nl, _ = gpu_list(same)
    assert (cg == 49).all()
    ro, co = oracle_list(same, method="brute")
    assert_same_lists(rg, cg, ro, co)
    nl.close()


def test_particles_on_both_faces_of_the_box():
    L = np.float32(12.0)
    r = 1.5
    pos = []
    for x in (0.0, np.nextafter(L, np.float32(0)), 6.0):
        for y in (0.0, 11.5, 6.0):
            for z in (0.25, 11.75, 6.0):
                pos.append([x, y, z])
    s = workloads.System(pos=np.array(pos, np.float32), types=np.zeros(len(pos), np.int32), L=L, n_types=1,
                         r_list=np.full((1, 1), r, np.float32), r_cut=np.full((1, 1), r, np.float32))
    rg, cg, nl, _ = gpu_list(s)
    ro, co = oracle_list(s, method="brute")
    assert_same_lists(rg, cg, ro, co)
    nl.close()


@pytest.mark.parametrize("traversal,wp", [(0, 32), (1, 32), (1, 16), (1, 8), (1, 4), (1, 1)])
def test_two_types_per_pair_cutoffs(traversal, wp):
    s = _uniform(20000, 30.0, 1.0, seed=5, n_types=3)
    s.r_list = np.array([[2.0, 2.5, 3.0], [2.5, 1.5, 0.0], [3.0, 0.0, 4.0]], np.float32)
    rg, cg, nl, _ = gpu_list(s, traversal=traversal, warp_particles=wp)
    ro, co = oracle_list(s)
    assert_same_lists(rg, cg, ro, co)
    t = nl.tree()
    o = oracle.lbvh_build(s.pos, s.types, [s.L] * 3, bundle_k=nl.get_option(1))
    assert np.array_equal(t["seg_start"].cpu().numpy(), o["seg_start"])
    assert np.array_equal(t["order"].cpu().numpy(), o["order"])
    nl.close()


def test_small_binary_mixture():
    s = workloads.binary_mixture(seed=3, L=40.0, n_large=20, n_small=25000)
    rg, cg, nl, _ = gpu_list(s, cap=512)
    ro, co = oracle_list(s, cap=512)
    assert_same_lists(rg, cg, ro, co)
    nl.close()


@pytest.mark.parametrize("wp,block", [(32, 256), (8, 256), (32, 64), (1, 128)])
def test_sparse_trees_walked_one_particle_per_warp(wp, block):
    # Types 1 and 2 are few and widely spaced (32 L^3 / count > (2 r_max)^3,
    # at most 4096 particles), so the kernel's leading blocks walk them one
    # particle per warp; type 1 has more particles than those blocks have
    # warps (152 SMs x 8), type 2 a single one, type 3 none.
    rng = np.random.default_rng(11)
    L = np.float32(60.0)
    counts = [60000, 3000, 1, 0]
    types = np.repeat(np.arange(4, dtype=np.int32), counts)
    types = types[rng.permutation(types.size)]
    pos = rng.uniform(0, L, size=(types.size, 3)).astype(np.float32)
    pos[pos >= L] = 0
    rl = np.array([[2.5, 4.0, 3.0, 2.0], [4.0, 6.0, 5.0, 2.0], [3.0, 5.0, 7.0, 2.0], [2.0, 2.0, 2.0, 2.0]],
                  np.float32)
    for t in (1, 2):
        assert 32 * float(L) ** 3 / counts[t] > (2 * rl[t].max()) ** 3
    s = workloads.System(pos=pos, types=types, L=L, n_types=4, r_list=rl, r_cut=rl.copy())
    rg, cg, nl, _ = gpu_list(s, warp_particles=wp, block=block)
    ro, co = oracle_list(s)
    assert_same_lists(rg, cg, ro, co)
    assert nl.max_count == int(co.max())
    nl.close()


def test_overflow_retry_and_truncation(cfg1):
    from paper_1901_08088_gb300 import _lib

    ro, co = oracle_list(cfg1, method="brute")
    rg, cg, nl, _ = gpu_list(cfg1, cap=8, max_retries=2)
    assert nl.cap >= co.max() and nl.cap % 32 == 0
    assert_same_lists(rg, cg, ro, co)
    nl.close()
    # no retries: counts complete, rows truncated at cap, overflow reported
    import torch

    from paper_1901_08088_gb300 import NeighborList

    nl = NeighborList(0)
    pos4 = torch.from_numpy(workloads.pack_float4(cfg1.pos, cfg1.types)).cuda()
    nl.build(pos4, cfg1.L)
    rc = nl.query(cfg1.r_list, cap=16, max_retries=0, raise_on_error=False)
    assert rc == _lib.QBVH_ERR_OVERFLOW
    rows, counts = nl.neighbors()
    counts = counts.cpu().numpy()
    assert np.array_equal(counts, co)
    rows = rows.cpu().numpy()
    sets = oracle.rows_as_sets(ro, co)
    for i in range(0, cfg1.n, 97):
        assert set(rows[i, :16].tolist()) <= sets[i]
    nl.close()


def test_radius_close_to_half_box():
    # the largest radius the library accepts: r just below (L/2)(1 - 2^-20)
    L = np.float32(8.0)
    r = np.float32(4.0 * (1 - 2.0 ** -19))
    s = _uniform(3000, float(L), float(r), seed=11)
    s.r_list[:] = r
    rg, cg, nl, _ = gpu_list(s, cap=2048)
    ro, co = oracle_list(s, cap=2048, method="brute")
    assert_same_lists(rg, cg, ro, co)
    nl.close()


def test_invalid_inputs_report_errors():
    import torch

    from paper_1901_08088_gb300 import NeighborList, _lib

    s = _uniform(1000, 10.0, 2.0, seed=9)
    nl = NeighborList(0)
    bad = s.pos.copy()
    bad[7, 1] = np.float32(10.0)       # == L: outside [0, L)
    nl.build(torch.from_numpy(workloads.pack_float4(bad, s.types)).cuda(), s.L)
    assert nl.query(2.0, raise_on_error=False) == _lib.QBVH_ERR_OUT_OF_BOX
    bad[7, 1] = np.float32(np.nan)
    nl.build(torch.from_numpy(workloads.pack_float4(bad, s.types)).cuda(), s.L)
    assert nl.query(2.0, raise_on_error=False) == _lib.QBVH_ERR_OUT_OF_BOX
    t = s.types.copy()
    t[3] = 5
    nl.build(torch.from_numpy(workloads.pack_float4(s.pos, t)).cuda(), s.L)
    assert nl.query(2.0, raise_on_error=False) == _lib.QBVH_ERR_BAD_TYPE
    nl.build(torch.from_numpy(workloads.pack_float4(s.pos, s.types)).cuda(), s.L)
    assert nl.query(5.0, raise_on_error=False) == _lib.QBVH_ERR_CUTOFF_TOO_LARGE
    assert nl.query(2.0, raise_on_error=False) == _lib.QBVH_OK
    # the traversal kernels are compiled for at most 256 threads per block
    assert _lib.lib().qbvh_set_option(nl.h, _lib.QBVH_OPT_QUERY_BLOCK, 512) == _lib.QBVH_ERR_INVALID_ARG
    assert _lib.lib().qbvh_set_option(nl.h, _lib.QBVH_OPT_QUERY_BLOCK, 48) == _lib.QBVH_ERR_INVALID_ARG
    nl.close()


@pytest.mark.parametrize("traversal,wp", [(0, 32), (1, 32), (1, 8)])
def test_candidate_mode_is_a_superset_with_few_false_positives(cfg1, traversal, wp):
    rg, cg, nl, _ = gpu_list(cfg1, candidates=1, cap=512, traversal=traversal, warp_particles=wp)
    ro, co = oracle_list(cfg1, method="brute")
    sets_o = oracle.rows_as_sets(ro, co)
    sets_g = oracle.rows_as_sets(rg, cg)
    extra = 0
    for i in range(cfg1.n):
        assert sets_o[i] <= sets_g[i]
        extra += len(sets_g[i]) - len(sets_o[i])
    # false positives stay a small fraction of the true neighbors (Sec. 4.1 reports ~5%)
    assert extra / co.sum() < 0.2
    nl.close()


def test_handle_reuse_across_sizes():
    from paper_1901_08088_gb300 import NeighborList
    import torch

    nl = NeighborList(0)
    for n in (5000, 300, 9000, 0, 40):
        s = _uniform(max(n, 1), 12.0, 2.2, seed=n)
        if n == 0:
            pos4 = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
            nl.build(pos4, 12.0)
            nl.query(2.2)
            assert nl.max_count == 0
            continue
        nl.build(torch.from_numpy(workloads.pack_float4(s.pos, s.types)).cuda(), s.L)
        nl.query(s.r_list)
        rows, counts = nl.neighbors()
        ro, co = oracle_list(s, method="brute")
        assert_same_lists(rows.cpu().numpy(), counts.cpu().numpy(), ro, co)
    nl.close()


@pytest.mark.slow
def test_full_size_binary_mixture():
    # 400 large + 395,280 small particles, per-type trees, per-pair radii 3.4 / 5.9 / 10.4
    s = workloads.workload("mixture_L100", seed=0)
    rg, cg, nl, _ = gpu_list(s, cap=512)
    ro, co = oracle_list(s, cap=512)
    assert_same_lists(rg, cg, ro, co)
    big = np.nonzero(s.types == 1)[0]
    assert cg[big].mean() > 100   # the large particles see their solvent shell
    nl.close()


@pytest.mark.slow
def test_spinodal_like_1m():
    # the inhomogeneous liquid/vapor stand-in of Sec. 4.3, N = 10^6, r_c = 3.0
    s = workloads.workload("spinodal_n1000000", seed=0)
    rg, cg, nl, _ = gpu_list(s, cap=256)
    ro, co = oracle_list(s, cap=256)
    assert np.array_equal(cg, co)
    idx = np.sort(np.random.default_rng(1).choice(s.n, 8192, replace=False))
    assert_same_lists(rg, cg, ro, co, idx=idx)
    nl.close()


@pytest.mark.parametrize("n_types", [1, 2, 4])
@pytest.mark.parametrize("n,K", [(2, 1), (3, 16), (33, 4), (1000, 16), (3072, 64), (3073, 32), (4096, 32)])
def test_small_system_tree_words_and_lists(n, K, n_types):
    # one system of at most 3072 particles is built by a single block, larger
    # ones by the multi-kernel build: the words of both must equal the
    # oracle's step-by-step construction, per type tree
    import torch

    L = max(6.0, (n / 0.5) ** (1 / 3))
    s = _uniform(n, L, 2.0, seed=7 * n + K, n_types=n_types)
    for node_format in (0, 1):
        rg, cg, nl, _ = gpu_list(s, bundle=K, node_format=node_format)
        ro, co = oracle_list(s, method="brute")
        assert_same_lists(rg, cg, ro, co)
        t = {k: v.cpu() for k, v in nl.tree().items()}
        o = oracle.lbvh_build(s.pos, s.types, [s.L] * n_types, bundle_k=K)
        assert np.array_equal(t["order"].numpy(), o["order"])
        assert np.array_equal(t["seg_start"].numpy(), o["seg_start"])
        assert np.array_equal(t["leaves"].view(torch.int32).numpy(), o["leaves"].view(np.int32))
        starts = o["seg_start"]
        for tr in range(n_types):   # internal slots of every tree but its last leaf's
            a, b = starts[tr], starts[tr + 1] - 1
            if b > a:
                assert np.array_equal(t["nodes"].numpy()[a:b], o["nodes"][a:b])
        # frames of the non-empty trees (an empty tree's frame is never read)
        full = np.diff(starts) > 0
        assert np.array_equal(t["frames"].numpy()[full, :6].view(np.int32), o["frame"][full].view(np.int32))
        nl.close()
