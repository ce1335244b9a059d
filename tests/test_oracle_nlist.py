"""Pins for the neighbor-list oracle (CPU only).

The oracle's brute force and cell list both implement the paper's problem
statement (Sec. 1, Fig. 1a; Sec. 4): every j != i within the list radius under
periodic boundaries.  They are pinned here against things other than
themselves: hand-derived lattice shells, an independent periodic k-d tree
(scipy), FP64 distances, and the invariants the definition implies
(symmetry, periodic-shift invariance, mean count rho * 4/3 pi r^3).
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _lattice(m, a):
    g = (np.arange(m, dtype=np.float64) + 0.5) * a
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.float32), np.float32(m * a)


@pytest.mark.parametrize("method", ["brute", "cell"])
def test_golden_lattice_shells(method):
    gold = json.load(open(os.path.join(GOLD, "lattice_shells.json")))
    for case in gold["cases"]:
        pos, L = _lattice(case["m"], case["a"])
        rows, counts = oracle.nlist(pos, L, case["r_list"], cap=128, method=method)
        assert (counts == case["count"]).all(), case
        # the neighbors are the shell sites themselves: check distances by FP64
        d = pos[rows[0, : counts[0]]].astype(np.float64) - pos[0]
        d -= float(L) * np.rint(d / float(L))
        assert (np.sqrt((d * d).sum(1)) < case["r_list"]).all()


def test_pair_across_boundary_and_self():
    L = np.float32(10.0)
    pos = np.array([[0.1, 5.0, 5.0], [9.8, 5.0, 5.0], [5.0, 5.0, 5.0]], np.float32)
    rows, counts = oracle.nlist(pos, L, 0.5, method="brute")
    assert counts.tolist() == [1, 1, 0]
    assert rows[0, 0] == 1 and rows[1, 0] == 0
    rows, counts = oracle.nlist(pos, L, 0.2, method="brute")
    assert counts.tolist() == [0, 0, 0]


def test_coincident_particles_are_neighbors_but_not_self():
    L = np.float32(8.0)
    pos = np.array([[1, 1, 1]] * 3 + [[5, 5, 5]], np.float32)
    rows, counts = oracle.nlist(pos, L, 1.0, method="brute")
    assert counts.tolist() == [2, 2, 2, 0]
    assert sorted(rows[0, :2].tolist()) == [1, 2]


def test_single_particle_has_empty_row():
    rows, counts = oracle.nlist(np.array([[1.0, 2.0, 3.0]], np.float32), np.float32(10), 3.0,
                                method="cell")
    assert counts.tolist() == [0]


def test_brute_equals_cell_list_configs():
    s = workloads.workload("lj_n4096_rho0.6")
    rb, cb = oracle.nlist(s.pos, s.L, s.r_list, method="brute")
    rc, cc = oracle.nlist(s.pos, s.L, s.r_list, method="cell")
    assert np.array_equal(cb, cc) and np.array_equal(rb, rc)
    # two types with unequal cutoffs
    rng = np.random.default_rng(7)
    L = np.float32(14.0)
    pos = rng.uniform(0, float(L), size=(3000, 3)).astype(np.float32)
    types = rng.integers(0, 2, 3000).astype(np.int32)
    rl = np.array([[1.5, 2.5], [2.5, 4.0]], np.float32)
    rb, cb = oracle.nlist(pos, L, rl, types, 2, method="brute")
    rc, cc = oracle.nlist(pos, L, rl, types, 2, method="cell")
    assert np.array_equal(cb, cc) and np.array_equal(rb, rc)


def test_matches_periodic_kdtree_outside_band():
    spatial = pytest.importorskip("scipy.spatial")
    s = workloads.jittered_lattice(6000, 0.7, 0.4, seed=3, r_cut=2.6, skin=0.3)
    rows, counts = oracle.nlist(s.pos, s.L, s.r_list, method="cell")
    r = float(s.r_list[0, 0])
    tree = spatial.cKDTree(s.pos.astype(np.float64), boxsize=float(s.L))
    inner = tree.query_ball_point(s.pos.astype(np.float64), r * (1 - 1e-6))
    outer = tree.query_ball_point(s.pos.astype(np.float64), r * (1 + 1e-6))
    sets = oracle.rows_as_sets(rows, counts)
    for i in range(s.n):
        lo = set(inner[i]) - {i}
        hi = set(outer[i]) - {i}
        assert lo <= sets[i] <= hi, i


def test_symmetry_exact():
    s = workloads.workload("lj_n4096_rho0.6")
    rows, counts = oracle.nlist(s.pos, s.L, s.r_list, method="cell")
    sets = oracle.rows_as_sets(rows, counts)
    for i in range(s.n):
        for j in sets[i]:
            assert i in sets[j]


def test_mean_count_near_ideal():
    s = workloads.workload("lj_n4096_rho0.6")
    _, counts = oracle.nlist(s.pos, s.L, s.r_list, method="cell")
    ideal = 0.6 * 4.0 / 3.0 * np.pi * float(s.r_list[0, 0]) ** 3
    assert abs(counts.mean() / ideal - 1) < 0.05


def test_fp64_band_check_clean_and_catches_planted_errors():
    s = workloads.workload("lj_n4096_rho0.6")
    rows, counts = oracle.nlist(s.pos, s.L, s.r_list, method="cell")
    nbad, _ = oracle.band_check(s.pos, s.L, s.r_list, rows, counts)
    assert nbad == 0
    # plant a missed neighbor and a spurious one in a copy of the list
    r2, c2 = rows.copy(), counts.copy()
    missing = r2[10, 0]
    r2[10, : c2[10] - 1] = r2[10, 1 : c2[10]]
    c2[10] -= 1
    far = int(np.argmax(((s.pos - s.pos[20]) ** 2).sum(1)))
    r2[20, c2[20]] = far
    c2[20] += 1
    nbad, bad = oracle.band_check(s.pos, s.L, s.r_list, r2, c2)
    assert nbad == 2
    assert (10, int(missing)) in bad and (20, far) in bad


def test_periodic_shift_invariance():
    s = workloads.workload("lj_n4096_rho0.6")
    rows, counts = oracle.nlist(s.pos, s.L, s.r_list, method="cell")
    shift = np.array([3.3, -7.1, 11.9])
    p2 = s.pos.astype(np.float64) + shift
    p2 = np.mod(p2, float(s.L)).astype(np.float32)
    p2[p2 >= s.L] = 0
    r2, c2 = oracle.nlist(p2, s.L, s.r_list, method="cell")
    a = oracle.rows_as_sets(rows, counts)
    b = oracle.rows_as_sets(r2, c2)
    r = float(s.r_list[0, 0])
    for i in range(s.n):
        for j in a[i] ^ b[i]:
            # a pair may only move across the boundary inside the FP32 rounding band
            d = s.pos[j].astype(np.float64) - s.pos[i]
            d -= float(s.L) * np.rint(d / float(s.L))
            assert abs(np.sqrt((d * d).sum()) - r) < 1e-5 * r


def test_cap_truncation_keeps_full_count():
    s = workloads.workload("lj_n4096_rho0.6")
    rows, counts = oracle.nlist(s.pos, s.L, s.r_list, cap=256, method="brute")
    r8, c8 = oracle.nlist(s.pos, s.L, s.r_list, cap=8, method="cell")
    assert np.array_equal(c8, counts)
    assert np.array_equal(r8, rows[:, :8])


def test_adversarial_pairs_at_radius_match_fp64_outside_band():
    # partners of particle 0 sit across the periodic boundary at r_list +- k ulp
    L = np.float32(20.0)
    r = np.float32(3.4)
    x0 = np.float32(19.0)
    centre = np.float32(np.float64(x0) + np.float64(r) - np.float64(L))   # ~2.4
    pts = [[x0, 10.0, 10.0]]
    for k in range(-400, 401, 8):
        x = centre
        step = np.float32(np.inf) if k > 0 else np.float32(-np.inf)
        for _ in range(abs(k)):
            x = np.nextafter(x, step, dtype=np.float32)
        pts.append([x, 10.0, 10.0])
    pos = np.array(pts, np.float32)
    rows, counts = oracle.nlist(pos, L, r, method="brute")
    nbad, bad = oracle.band_check(pos, L, r, rows, counts, band=1e-6)
    assert nbad == 0, bad
    row0 = set(rows[0, : counts[0]].tolist())
    # 400 ulp closer is inside, 400 ulp farther is outside
    assert 1 in row0 and len(pts) - 1 not in row0


@pytest.mark.parametrize("method", ["brute", "cell"])
def test_types_do_not_matter_when_every_pair_has_one_radius(method):
    # The definition selects j by d2 < r(t_i, t_j)^2 only, so with one radius
    # for every type pair the typed list equals the list of the same positions
    # with every type 0 (the property one tree per system relies on), and a
    # zero radius for one pair removes exactly that pair's entries.
    s = workloads.two_type_lj(seed=3, n_sys=1, n=3000)[0]
    r = float(s.r_list[0, 0])
    rt, ct = oracle.nlist(s.pos, s.L, np.full((2, 2), r, np.float32), s.types, 2, method=method)
    r1, c1 = oracle.nlist(s.pos, s.L, r, method=method)
    assert np.array_equal(ct, c1)
    assert np.array_equal(rt, r1)
    rz, cz = oracle.nlist(s.pos, s.L, np.array([[r, r], [r, 0.0]], np.float32), s.types, 2, method=method)
    sets1 = oracle.rows_as_sets(r1, c1)
    setsz = oracle.rows_as_sets(rz, cz)
    for i in range(0, s.n, 7):
        keep = {j for j in sets1[i] if not (s.types[i] == 1 and s.types[j] == 1)}
        assert setsz[i] == keep
