"""GPU parity for double-precision particle data (Sec. 2.2, Sec. 4.1-4.2).

The tree is built over outward-rounded FP32 boxes of the FP64 positions, the
traversal runs in FP32, and the leaf decision is the pinned FP64 expression
(FP32 outside a proven band around r^2).  Every list is compared bit-exactly,
as sets, with the FP64 oracle on the same seeded positions.
"""
import numpy as np
import pytest

import oracle
import workloads
from helpers import assert_same_lists

pytestmark = pytest.mark.gpu


def gpu_list64(s, cap=256, bundle=None, node_format=None, block=None, max_retries=4):
    import torch

    from paper_1901_08088_gb300 import NeighborList, _lib

    nl = NeighborList(0)
    if bundle is not None:
        nl.set_option(_lib.QBVH_OPT_BUNDLE, bundle)
    if node_format is not None:
        nl.set_option(_lib.QBVH_OPT_NODE_FORMAT, node_format)
    if block is not None:
        nl.set_option(_lib.QBVH_OPT_QUERY_BLOCK, block)
    pos = torch.from_numpy(workloads.pack_double4(s.pos, s.types)).cuda()
    nl.build_f64(pos, s.L, s.n_types)
    nl.query(s.r_list, cap=cap, max_retries=max_retries)
    rows, counts = nl.neighbors()
    return rows.cpu().numpy(), counts.cpu().numpy(), nl


def _uniform64(n, L, r, seed, n_types=1):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, L, size=(n, 3))
    pos[pos >= L] = 0.0
    types = rng.integers(0, n_types, n).astype(np.int32)
    rl = np.full((n_types, n_types), r, np.float32)
    return workloads.System64(pos=pos, types=types, L=float(L), n_types=n_types, r_list=rl, r_cut=rl.copy())


@pytest.fixture(scope="module")
def cfg1_64():
    return workloads.jittered_lattice64(4096, 0.6, 0.3, seed=0, r_cut=3.0, skin=0.4)


@pytest.mark.parametrize("node_format", [0, 1])
@pytest.mark.parametrize("bundle", [1, 4, 16, 32])
def test_config1_fp64_equals_bruteforce(cfg1_64, bundle, node_format):
    rg, cg, nl = gpu_list64(cfg1_64, bundle=bundle, node_format=node_format)
    ro, co = oracle.nlist64(cfg1_64.pos, cfg1_64.L, cfg1_64.r_list, method="brute")
    assert_same_lists(rg, cg, ro, co)
    assert nl.max_count == co.max()
    nl.close()


@pytest.mark.parametrize("n", [1, 2, 33, 4097, 12345])
def test_ragged_sizes_fp64(n):
    L = max(8.0, (n / 0.5) ** (1 / 3))
    s = _uniform64(n, L, 2.5, seed=n)
    rg, cg, nl = gpu_list64(s, block=64 if n % 2 else 256)
    ro, co = oracle.nlist64(s.pos, s.L, s.r_list, method="brute")
    assert_same_lists(rg, cg, ro, co)
    nl.close()


def test_two_types_fp64():
    s = _uniform64(6000, 16.0, 1.0, seed=3, n_types=2)
    s.r_list = np.array([[1.5, 2.5], [2.5, 3.9]], np.float32)
    rg, cg, nl = gpu_list64(s, cap=512)
    ro, co = oracle.nlist64(s.pos, s.L, s.r_list, s.types, 2, cap=512)
    assert_same_lists(rg, cg, ro, co)
    nl.close()


@pytest.mark.parametrize("rho", [0.2, 0.8])
@pytest.mark.parametrize("kind", ["wca", "lj"])
def test_paper_state_points_fp64(kind, rho):
    # Sec. 4.1-4.2: N = 128,000 in double precision, r_c = 3.0 (LJ) or 2^(1/6) (WCA)
    rc = 3.0 if kind == "lj" else workloads.WCA_RCUT
    s = workloads.jittered_lattice64(128_000, rho, 0.3, seed=2, r_cut=rc, skin=0.0)
    rg, cg, nl = gpu_list64(s)
    ro, co = oracle.nlist64(s.pos, s.L, s.r_list)
    assert_same_lists(rg, cg, ro, co)
    nl.close()


def test_pairs_closer_than_fp32_resolution_at_the_radius():
    # partners at r +- k 2^-40 across the periodic boundary and in the box:
    # their FP32-rounded distances cannot tell them apart, so only the FP64
    # decision inside the band lists the inner ones and not the outer ones
    L = 20.0
    r = float(np.float32(3.4))
    pts = [[19.0, 10.0, 10.0], [5.0, 5.0, 5.0]]
    ks = [-4096, -64, -8, -1, 1, 8, 64, 4096]
    for k in ks:
        pts.append([19.0 + r + k * 2.0 ** -40 - L, 10.0, 10.0])     # across the x face
    for k in ks:
        pts.append([5.0, 5.0 + r + k * 2.0 ** -40, 5.0])           # inside the box
    pos = np.array(pts, np.float64)
    s = workloads.System64(pos=pos, types=np.zeros(len(pts), np.int32), L=L, n_types=1,
                           r_list=np.full((1, 1), np.float32(3.4)), r_cut=np.full((1, 1), np.float32(3.4)))
    rg, cg, nl = gpu_list64(s)
    ro, co = oracle.nlist64(s.pos, s.L, s.r_list, method="brute")
    assert_same_lists(rg, cg, ro, co)
    sets = oracle.rows_as_sets(rg, cg)
    inner_x = {2 + t for t, k in enumerate(ks) if k < 0}
    inner_y = {2 + len(ks) + t for t, k in enumerate(ks) if k < 0}
    assert inner_x <= sets[0] and not ({2 + t for t, k in enumerate(ks) if k > 0} & sets[0])
    assert inner_y <= sets[1] and not ({2 + len(ks) + t for t, k in enumerate(ks) if k > 0} & sets[1])
    nl.close()


def test_fp64_inputs_are_validated():
    import torch

    from paper_1901_08088_gb300 import NeighborList, _lib, qbvh

    s = _uniform64(1000, 10.0, 2.0, seed=9)
    nl = NeighborList(0)
    bad = workloads.pack_double4(s.pos, s.types)
    bad[7, 1] = 10.0                    # == L: outside [0, L)
    nl.build_f64(torch.from_numpy(bad).cuda(), s.L)
    assert nl.query(2.0, raise_on_error=False) == _lib.QBVH_ERR_OUT_OF_BOX
    bad[7, 1] = np.nan
    nl.build_f64(torch.from_numpy(bad).cuda(), s.L)
    assert nl.query(2.0, raise_on_error=False) == _lib.QBVH_ERR_OUT_OF_BOX
    bad = workloads.pack_double4(s.pos, s.types)
    bad[3, 3] = 0.5                     # type not a whole number
    nl.build_f64(torch.from_numpy(bad).cuda(), s.L)
    assert nl.query(2.0, raise_on_error=False) == _lib.QBVH_ERR_BAD_TYPE
    good = torch.from_numpy(workloads.pack_double4(s.pos, s.types)).cuda()
    nl.build_f64(good, s.L)
    assert nl.query(2.0, raise_on_error=False) == _lib.QBVH_OK
    assert nl.query(5.0, raise_on_error=False) == _lib.QBVH_ERR_CUTOFF_TOO_LARGE
    # 16-byte aligned only: refused before any launch
    flat = torch.zeros(4 * 1001 + 2, dtype=torch.float64, device="cuda")
    assert qbvh.qbvh_build_f64(nl.h, flat[2:].view(1001, 4), 10.0) == _lib.QBVH_ERR_INVALID_ARG
    # the candidate mode and the grid method take FP32 data only
    nl.build_f64(good, s.L)
    nl.set_option(_lib.QBVH_OPT_CANDIDATES, 1)
    assert nl.query(2.0, raise_on_error=False) == _lib.QBVH_ERR_INVALID_ARG
    nl.set_option(_lib.QBVH_OPT_CANDIDATES, 0)
    nl.set_option(_lib.QBVH_OPT_METHOD, 1)
    assert qbvh.qbvh_build_f64(nl.h, good, s.L) == _lib.QBVH_ERR_INVALID_ARG
    nl.close()


def test_fp32_build_after_fp64_build_on_one_handle(cfg1_64):
    import torch

    from paper_1901_08088_gb300 import NeighborList

    nl = NeighborList(0)
    nl.build_f64(torch.from_numpy(workloads.pack_double4(cfg1_64.pos, cfg1_64.types)).cuda(), cfg1_64.L)
    nl.query(cfg1_64.r_list)
    s32 = workloads.workload("lj_n4096_rho0.6")
    nl.build(torch.from_numpy(workloads.pack_float4(s32.pos, s32.types)).cuda(), s32.L)
    nl.query(s32.r_list)
    rows, counts = nl.neighbors()
    ro, co = oracle.nlist(s32.pos, s32.L, s32.r_list, method="brute")
    assert_same_lists(rows.cpu().numpy(), counts.cpu().numpy(), ro, co)
    nl.close()


@pytest.mark.slow
def test_full_size_fp64_2m():
    s = workloads.jittered_lattice64(2_097_152, 0.8, 0.25, seed=0, r_cut=3.0, skin=0.3)
    rg, cg, nl = gpu_list64(s)
    ro, co = oracle.nlist64(s.pos, s.L, s.r_list)
    assert np.array_equal(cg, co)
    idx = np.sort(np.random.default_rng(0).choice(s.n, 8192, replace=False))
    assert_same_lists(rg, cg, ro, co, idx=idx)
    nl.close()


@pytest.mark.slow
def test_spinodal_like_1m_fp64():
    s = workloads.spinodal_like(1_000_000, 0.2, seed=0, double=True)
    rg, cg, nl = gpu_list64(s)
    ro, co = oracle.nlist64(s.pos, s.L, s.r_list)
    assert np.array_equal(cg, co)
    idx = np.sort(np.random.default_rng(1).choice(s.n, 8192, replace=False))
    assert_same_lists(rg, cg, ro, co, idx=idx)
    nl.close()
