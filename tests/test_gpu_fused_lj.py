"""Traversal and Lennard-Jones forward in one call (qbvh_query_lj_async).

For one system of one type the traversal itself sums the truncated and
shifted pair terms of Eq. 1 for every pair it accepts.  Checked through the
C ABI: the list it writes equals the plain query's and the oracle's (bit for
bit), and the energy, forces and eps/sigma gradients agree with the FP64
oracle within 1e-5 relative (forces normwise, as for the list pass), on the
bench workload's options, under every node format and bundle size, for
particles whose neighbours lie across a box face, and when the call falls
back to the two passes (two types, other mappings).
"""
import numpy as np
import pytest

import oracle
import workloads
from helpers import assert_same_lists, assert_same_lists_chunked, gpu_list, oracle_list

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _fused(s, E, S, rc, cap=256, fused=1, **opts):
    """Build, then one qbvh_query_lj_async call; returns rows, counts, status and the LJ outputs.
    fused=1 turns on the LJ terms inside the traversal (QBVH_OPT_FUSED_LJ)."""
    import torch

    from paper_1901_08088_gb300 import NeighborList, _lib

    names = {"bundle": _lib.QBVH_OPT_BUNDLE, "block": _lib.QBVH_OPT_QUERY_BLOCK,
             "node_format": _lib.QBVH_OPT_NODE_FORMAT, "warp_particles": _lib.QBVH_OPT_WARP_PARTICLES,
             "traversal": _lib.QBVH_OPT_TRAVERSAL}
    nl = NeighborList(0)
    for k, v in opts.items():
        nl.set_option(names[k], v)
    nl.set_option(_lib.QBVH_OPT_FUSED_LJ, fused)
    T = s.n_types
    pos4 = torch.from_numpy(workloads.pack_float4(s.pos, s.types)).cuda()
    nl.build(pos4, s.L, T)
    eps = torch.tensor(np.asarray(E, np.float32), device="cuda")
    sig = torch.tensor(np.asarray(S, np.float32), device="cuda")
    n = s.n
    e = torch.full((n,), np.nan, dtype=torch.float32, device="cuda")
    U = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    F = torch.full((n, 3), np.nan, dtype=torch.float32, device="cuda")
    dE = torch.full((1, T, T), np.nan, dtype=torch.float64, device="cuda")
    dS = torch.full((1, T, T), np.nan, dtype=torch.float64, device="cuda")
    nl.query_lj_async(pos4, s.r_list, cap, eps, sig, rc, e, U, F, dE, dS)
    torch.cuda.synchronize()
    status, _ = nl.query_status()
    rows, counts = nl.neighbors()
    out = dict(rows=rows.cpu().numpy(), counts=counts.cpu().numpy(), status=status, e=e.cpu().numpy(),
               U=U.cpu().numpy(), F=F.cpu().numpy(), dE=dE.cpu().numpy()[0], dS=dS.cpu().numpy()[0])
    return out, nl


def _check_vs_oracle(out, s, E, S, rc, ro, co):
    ref = oracle.lj_fp64(s.pos, s.types, s.L, E, S, np.full((s.n_types, s.n_types), rc, np.float32), ro, co)
    assert abs(out["U"][0] - ref["U"]) <= TOL * abs(ref["U"]), (out["U"][0], ref["U"])
    assert _rel(out["F"], ref["F"]) <= TOL
    assert _rel(out["e"], ref["e"]) <= TOL
    for a in range(s.n_types):
        for b in range(s.n_types):
            assert abs(out["dE"][a, b] - ref["dE"][a, b]) <= TOL * abs(ref["dE"][a, b]), (a, b)
            assert abs(out["dS"][a, b] - ref["dS"][a, b]) <= TOL * abs(ref["dS"][a, b]), (a, b)
    return ref


@pytest.mark.parametrize("node_format", [0, 1, 2])
@pytest.mark.parametrize("bundle", [1, 16, 64])
def test_fused_lj_config1_vs_fp64_oracle(node_format, bundle):
    s = workloads.workload("lj_n4096_rho0.6", seed=11)
    out, nl = _fused(s, [[1.0]], [[1.0]], 3.0, node_format=node_format, bundle=bundle)
    assert out["status"] == 0
    ro, co = oracle_list(s, method="brute")
    assert_same_lists(out["rows"], out["counts"], ro, co)
    _check_vs_oracle(out, s, [[1.0]], [[1.0]], 3.0, ro, co)
    nl.close()


def test_fused_matches_two_passes_and_repeats_bit_for_bit():
    """The fused sums agree with the separate pass to FP32 rounding; two fused
    calls give identical bits (fixed summation order)."""
    from paper_1901_08088_gb300 import _lib

    s = workloads.workload("lj_n4096_rho0.6", seed=12)
    a, nl_a = _fused(s, [[1.2]], [[0.95]], 2.7)
    b, nl_b = _fused(s, [[1.2]], [[0.95]], 2.7)
    c, nl_c = _fused(s, [[1.2]], [[0.95]], 2.7, fused=0)
    assert nl_c.get_option(_lib.QBVH_OPT_FUSED_LJ) == 0
    for k in ("U", "F", "e", "dE", "dS"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["counts"], c["counts"])
    assert abs(a["U"][0] - c["U"][0]) <= 1e-6 * abs(c["U"][0])
    assert _rel(a["F"], c["F"]) <= 1e-6
    assert abs(a["dS"][0, 0] - c["dS"][0, 0]) <= 1e-6 * abs(c["dS"][0, 0])
    for nl in (nl_a, nl_b, nl_c):
        nl.close()


@pytest.mark.parametrize("n,rho,rc", [(2, 0.01, 1.2), (31, 0.8, 1.0), (33, 0.8, 1.0), (1000, 0.8, 2.5),
                                      (12345, 0.8, 2.5)])
def test_fused_lj_ragged_sizes_and_box_faces(n, rho, rc):
    """Ragged warps and blocks; small boxes, so that many pairs cross a face
    (image pairs take the once-rounded difference, as the list pass does)."""
    s = workloads.jittered_lattice(n, rho, 0.3, seed=n, r_cut=rc, skin=0.3)
    assert s.L > 2 * float(s.r_list.max()) * (1 + 1e-6)
    out, nl = _fused(s, [[1.0]], [[1.0]], rc)
    assert out["status"] == 0
    ro, co = oracle_list(s, method="brute")
    assert_same_lists(out["rows"], out["counts"], ro, co)
    if co.sum() > 0:
        _check_vs_oracle(out, s, [[1.0]], [[1.0]], rc, ro, co)
    else:
        assert out["U"][0] == 0.0 and not out["F"].any()
    nl.close()


def test_fused_lj_mappings_that_fall_back():
    """One particle per lane is the fused walk; other mappings and two types run
    the traversal and the list pass back to back through the same call."""
    s = workloads.workload("lj_n4096_rho0.6", seed=13)
    ro, co = oracle_list(s, method="brute")
    for opts in ({"warp_particles": 4}, {"traversal": 0}):
        out, nl = _fused(s, [[1.0]], [[1.0]], 3.0, **opts)
        assert out["status"] == 0
        assert_same_lists(out["rows"], out["counts"], ro, co)
        _check_vs_oracle(out, s, [[1.0]], [[1.0]], 3.0, ro, co)
        nl.close()
    t = workloads.two_type_lj(seed=5, n_sys=1, n=6000)[0]
    out, nl = _fused(t, t.meta["eps"], t.meta["sig"], 2.5)
    ro, co = oracle_list(t)
    assert_same_lists(out["rows"], out["counts"], ro, co)
    _check_vs_oracle(out, t, t.meta["eps"], t.meta["sig"], 2.5, ro, co)
    nl.close()


def test_fused_lj_overflow_keeps_every_pair():
    """Rows past cap are truncated and the status says OVERFLOW; the fused sums
    still cover every pair of the full list."""
    from paper_1901_08088_gb300 import _lib

    s = workloads.workload("lj_n4096_rho0.6", seed=14)
    out, nl = _fused(s, [[1.0]], [[1.0]], 3.0, cap=40)
    assert out["status"] == _lib.QBVH_ERR_OVERFLOW
    ro, co = oracle_list(s, method="brute")
    assert np.array_equal(out["counts"], co)
    _check_vs_oracle(out, s, [[1.0]], [[1.0]], 3.0, ro, co)
    nl.close()


def test_fused_lj_invalid_arguments():
    import torch

    from paper_1901_08088_gb300 import _lib
    from paper_1901_08088_gb300.qbvh import qbvh_query_lj_async

    s = workloads.workload("lj_n4096_rho0.6", seed=15)
    _, _, nl, pos4 = gpu_list(s)
    one = torch.ones((1, 1), dtype=torch.float32, device="cuda")
    U = torch.empty(1, dtype=torch.float64, device="cuda")
    # r_cut above the list radius, and no energy output
    assert qbvh_query_lj_async(nl.h, pos4, 3.4, 1, 256, one, one, 3.5, None, U, None, None, None) == \
        _lib.QBVH_ERR_INVALID_ARG
    assert qbvh_query_lj_async(nl.h, pos4, 3.4, 1, 256, one, one, 3.0, None, None, None, None, None) == \
        _lib.QBVH_ERR_INVALID_ARG
    nl.close()


@pytest.mark.slow
@pytest.mark.parametrize("node_format", [0, 1])
def test_fused_lj_bench_workload_full_size(node_format):
    """N = 2,097,152 at the bench's options (K = 64, 128-thread blocks): every
    row equals the cell-list oracle, and E, F, gradients are within 1e-5 of FP64."""
    import torch

    s = workloads.workload("lj_n2097152_rho0.8", seed=0)
    out, nl = _fused(s, [[1.0]], [[1.0]], 3.0, node_format=node_format, bundle=64, block=128)
    assert out["status"] == 0
    ro, co = oracle_list(s)
    rows_dev, _ = nl.neighbors()
    assert_same_lists_chunked(rows_dev, out["counts"], ro, co)
    ref = _check_vs_oracle(out, s, [[1.0]], [[1.0]], 3.0, ro, co)
    print(f"fused LJ at N = 2M vs FP64: U {abs(out['U'][0] - ref['U']) / abs(ref['U']):.2e}, "
          f"F {_rel(out['F'], ref['F']):.2e}")
    nl.close()
    torch.cuda.empty_cache()
