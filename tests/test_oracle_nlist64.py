"""Pins for the double-precision neighbor-list oracle (CPU only).

The FP64 oracle lists, for particle data kept in double precision (Sec. 2.2),
every j != i within the list radius under periodic boundaries, decided by one
pinned FP64 minimum-image expression.  It is pinned against things other than
itself: an independent periodic k-d tree (scipy) on the same FP64 data, the
FP32 oracle on data that FP32 represents exactly, hand-placed pairs across the
boundary, and the invariants of the definition (symmetry, periodic-shift
invariance, mean count rho * 4/3 pi r^3).
"""
import numpy as np
import pytest

import oracle
import workloads


def _uniform64(n, L, seed, n_types=1):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, L, size=(n, 3))
    pos[pos >= L] = 0.0
    types = rng.integers(0, n_types, n).astype(np.int32)
    return pos, types


def test_pair_across_boundary_self_and_coincident():
    L = 10.0
    pos = np.array([[0.1, 5, 5], [9.8, 5, 5], [5, 5, 5], [5, 5, 5]], np.float64)
    rows, counts = oracle.nlist64(pos, L, 0.5, method="brute")
    assert counts.tolist() == [1, 1, 1, 1]
    assert rows[0, 0] == 1 and rows[1, 0] == 0 and rows[2, 0] == 3 and rows[3, 0] == 2
    rows, counts = oracle.nlist64(pos, L, 0.2, method="brute")
    assert counts.tolist() == [0, 0, 1, 1]


@pytest.mark.parametrize("n", [1, 2, 33, 4000])
def test_brute_equals_cell_list(n):
    pos, types = _uniform64(n, 13.0, seed=n, n_types=2)
    rl = np.array([[1.5, 2.5], [2.5, 3.9]], np.float32)
    rb, cb = oracle.nlist64(pos, 13.0, rl, types, 2, method="brute")
    rc, cc = oracle.nlist64(pos, 13.0, rl, types, 2, method="cell")
    assert np.array_equal(cb, cc) and np.array_equal(rb, rc)


def test_matches_periodic_kdtree_outside_band():
    spatial = pytest.importorskip("scipy.spatial")
    s = workloads.jittered_lattice64(6000, 0.7, 0.4, seed=3, r_cut=2.6, skin=0.3)
    rows, counts = oracle.nlist64(s.pos, s.L, s.r_list, method="cell")
    r = float(s.r_list[0, 0])
    tree = spatial.cKDTree(s.pos, boxsize=s.L)
    inner = tree.query_ball_point(s.pos, r * (1 - 1e-12))
    outer = tree.query_ball_point(s.pos, r * (1 + 1e-12))
    sets = oracle.rows_as_sets(rows, counts)
    for i in range(s.n):
        lo = set(inner[i]) - {i}
        hi = set(outer[i]) - {i}
        assert lo <= sets[i] <= hi, i


def test_wca_cutoff_matches_kdtree():
    # the WCA fluid's cutoff 2^(1/6) sigma (Sec. 4.2), no skin, both densities
    spatial = pytest.importorskip("scipy.spatial")
    for rho in (0.2, 0.8):
        s = workloads.jittered_lattice64(8000, rho, 0.4, seed=5, r_cut=workloads.WCA_RCUT, skin=0.0)
        rows, counts = oracle.nlist64(s.pos, s.L, s.r_list, method="cell")
        r = float(s.r_list[0, 0])
        tree = spatial.cKDTree(s.pos, boxsize=s.L)
        inner = tree.query_ball_point(s.pos, r * (1 - 1e-12))
        outer = tree.query_ball_point(s.pos, r * (1 + 1e-12))
        sets = oracle.rows_as_sets(rows, counts)
        for i in range(s.n):
            assert set(inner[i]) - {i} <= sets[i] <= set(outer[i]) - {i}, (rho, i)


def test_symmetry_exact():
    s = workloads.jittered_lattice64(4096, 0.6, 0.3, seed=0, r_cut=3.0, skin=0.4)
    rows, counts = oracle.nlist64(s.pos, s.L, s.r_list, method="cell")
    sets = oracle.rows_as_sets(rows, counts)
    for i in range(s.n):
        for j in sets[i]:
            assert i in sets[j]


def test_mean_count_near_ideal():
    pos, _ = _uniform64(20000, 25.0, seed=2)
    _, counts = oracle.nlist64(pos, 25.0, 2.0, method="cell")
    ideal = 20000 / 25.0 ** 3 * 4.0 / 3.0 * np.pi * 2.0 ** 3
    assert abs(counts.mean() / ideal - 1) < 0.02


def test_periodic_shift_invariance():
    s = workloads.jittered_lattice64(4096, 0.6, 0.3, seed=1, r_cut=3.0, skin=0.4)
    r = float(s.r_list[0, 0])
    rows, counts = oracle.nlist64(s.pos, s.L, s.r_list)
    shift = np.random.default_rng(4).uniform(0, s.L, 3)
    moved = np.mod(s.pos + shift, s.L)
    moved[moved >= s.L] = 0.0
    rows2, counts2 = oracle.nlist64(moved, s.L, s.r_list)
    a, b = oracle.rows_as_sets(rows, counts), oracle.rows_as_sets(rows2, counts2)
    # re-rounding moves pairs only within a relative 1e-12 of the radius
    for i in range(s.n):
        for j in a[i] ^ b[i]:
            d = s.pos[j] - s.pos[i]
            d -= s.L * np.rint(d / s.L)
            assert abs(np.sqrt((d * d).sum()) - r) < 1e-12 * r, (i, j)


def test_agrees_with_fp32_oracle_on_fp32_data():
    # positions FP32 represents exactly and an FP32 box: both decisions
    # approximate the same real distance, so they differ only within a
    # relative 1e-6 of the radius
    s = workloads.workload("lj_n4096_rho0.6")
    r32, c32 = oracle.nlist(s.pos, s.L, s.r_list)
    r64, c64 = oracle.nlist64(s.pos.astype(np.float64), float(s.L), s.r_list)
    a, b = oracle.rows_as_sets(r32, c32), oracle.rows_as_sets(r64, c64)
    r = float(s.r_list[0, 0])
    L = float(s.L)
    p = s.pos.astype(np.float64)
    for i in range(s.n):
        for j in a[i] ^ b[i]:
            d = p[j] - p[i]
            d -= L * np.rint(d / L)
            assert abs(np.sqrt((d * d).sum()) - r) < 1e-6 * r, (i, j)


def test_hand_placed_pairs_at_the_radius():
    # partners of particle 0 across the boundary at r +- k * 2^-40 (far above
    # FP64 resolution, far below FP32's): inside pairs listed, outside not
    L = 20.0
    r = float(np.float32(3.4))
    x0 = 19.0
    pts = [[x0, 10.0, 10.0]]
    ks = [-64, -8, -1, 1, 8, 64]
    for k in ks:
        pts.append([x0 + r + k * 2.0 ** -40 - L, 10.0, 10.0])
    pos = np.array(pts, np.float64)
    rows, counts = oracle.nlist64(pos, L, np.float32(3.4), method="brute")
    row0 = set(rows[0, : counts[0]].tolist())
    assert row0 == {1 + t for t, k in enumerate(ks) if k < 0}
