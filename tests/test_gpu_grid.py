"""GPU parity of the uniform-grid comparator (the paper's sort-based cell list,
Sec. 3): the same exact list as the oracle, for every lanes-per-particle
setting, ragged sizes, several types with per-pair radii, and overflow."""
import numpy as np
import pytest

import workloads
from helpers import assert_same_lists, gpu_list, oracle_list

pytestmark = pytest.mark.gpu


def _uniform(n, L, r, seed, n_types=1):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, L, size=(n, 3)).astype(np.float32)
    pos[pos >= np.float32(L)] = 0
    types = rng.integers(0, n_types, n).astype(np.int32)
    rl = np.full((n_types, n_types), r, np.float32)
    return workloads.System(pos=pos, types=types, L=np.float32(L), n_types=n_types, r_list=rl, r_cut=rl.copy())


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_grid_config1_equals_bruteforce(lanes):
    s = workloads.workload("lj_n4096_rho0.6", seed=0)
    rg, cg, nl, _ = gpu_list(s, method=1, grid_lanes=lanes)
    ro, co = oracle_list(s, method="brute")
    assert_same_lists(rg, cg, ro, co)
    assert nl.max_count == co.max()
    nl.close()


@pytest.mark.parametrize("n", [1, 2, 33, 4097, 20000])
def test_grid_ragged_sizes(n):
    L = max(9.0, (n / 0.5) ** (1 / 3))
    s = _uniform(n, L, 2.5, seed=n)
    rg, cg, nl, _ = gpu_list(s, method=1, grid_lanes=4)
    ro, co = oracle_list(s, method="brute")
    assert_same_lists(rg, cg, ro, co)
    nl.close()


def test_grid_types_and_small_radius():
    s = _uniform(20000, 30.0, 1.0, seed=5, n_types=3)
    s.r_list = np.array([[2.0, 2.5, 3.0], [2.5, 1.5, 0.0], [3.0, 0.0, 4.0]], np.float32)
    rg, cg, nl, _ = gpu_list(s, method=1)
    ro, co = oracle_list(s)
    assert_same_lists(rg, cg, ro, co)
    nl.close()
    # a radius much smaller than the mean spacing: the cell count is capped
    t = _uniform(5000, 40.0, 0.3, seed=6)
    rg, cg, nl, _ = gpu_list(t, method=1)
    ro, co = oracle_list(t, method="brute")
    assert_same_lists(rg, cg, ro, co)
    nl.close()


def test_grid_overflow_retry():
    s = workloads.workload("lj_n4096_rho0.6", seed=2)
    rg, cg, nl, _ = gpu_list(s, method=1, cap=8, max_retries=2)
    ro, co = oracle_list(s, method="brute")
    assert_same_lists(rg, cg, ro, co)
    nl.close()


@pytest.mark.slow
def test_grid_full_size_matches_bvh():
    s = workloads.workload("lj_n2097152_rho0.8", seed=0)
    rb, cb, nl, _ = gpu_list(s)
    rgd, cgd, nl2, _ = gpu_list(s, method=1)
    assert np.array_equal(cb, cgd)
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(s.n, 20000, replace=False))
    assert_same_lists(rb, cb, rgd, cgd, idx=idx)
    nl.close()
    nl2.close()
