"""GPU parity of the batched many-system build + query: every system's rows
equal the oracle's list of that system alone, and the per-system trees equal
the oracle's segmented construction."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import assert_same_lists, concat, oracle_list

pytestmark = pytest.mark.gpu


def _batched(systems, n_types=1, cap=256, r=None, traversal=None, wp=None):
    import torch

    from paper_1901_08088_gb300 import NeighborList, _lib

    pos4, off, Ls = concat(systems)
    nl = NeighborList(0)
    if traversal is not None:
        nl.set_option(_lib.QBVH_OPT_TRAVERSAL, traversal)
    if wp is not None:
        nl.set_option(_lib.QBVH_OPT_WARP_PARTICLES, wp)
    nl.build_batched(torch.from_numpy(pos4).cuda(), off, Ls, n_types=n_types)
    nl.query(systems[0].r_list if r is None else r, cap=cap)
    rows, counts = nl.neighbors()
    return rows.cpu().numpy(), counts.cpu().numpy(), off, nl


def _check_systems(systems, rows, counts, off):
    for k, s in enumerate(systems):
        a, b = off[k], off[k + 1]
        ro, co = oracle_list(s, method="brute" if s.n < 3000 else "cell")
        # batched rows hold indices into the concatenated array
        assert_same_lists(rows[a:b] - a, counts[a:b], ro, co)


@pytest.mark.parametrize("traversal,wp", [(0, 32), (1, 32), (1, 16), (1, 8), (1, 2), (1, 1)])
def test_small_ensemble_matches_oracle_per_system(traversal, wp):
    systems = workloads.batched_ensemble(seed=5, n_sys=12, n_min=250, n_max=3000)
    rows, counts, off, nl = _batched(systems, traversal=traversal, wp=wp)
    _check_systems(systems, rows, counts, off)
    nl.close()


def test_segmented_trees_equal_oracle():
    import torch

    systems = workloads.batched_ensemble(seed=6, n_sys=5, n_min=200, n_max=2000)
    rows, counts, off, nl = _batched(systems)
    t = {k: v.cpu() for k, v in nl.tree().items()}
    seg = np.concatenate([np.full(s.n, k, np.int32) for k, s in enumerate(systems)])
    pos = np.concatenate([s.pos for s in systems])
    Ls = np.array([s.L for s in systems], np.float32)
    o = oracle.lbvh_build(pos, seg, Ls, bundle_k=nl.get_option(1))
    assert np.array_equal(t["order"].numpy(), o["order"])
    assert np.array_equal(t["seg_start"].numpy(), o["seg_start"])
    assert np.array_equal(t["leaves"].view(torch.int32).numpy(), o["leaves"].view(np.int32))
    nodes = t["nodes"].numpy()
    for k in range(len(systems)):
        a, b = o["seg_start"][k], o["seg_start"][k + 1] - 1
        assert np.array_equal(nodes[a:b], o["nodes"][a:b])
    nl.close()


def test_ensemble_with_empty_and_single_particle_systems():
    base = workloads.batched_ensemble(seed=7, n_sys=4, n_min=250, n_max=900)
    one = workloads.jittered_lattice(1, 0.001, 0.1, seed=1, r_cut=2.5, skin=0.3)
    systems = [base[0], one, base[1], base[2], one, base[3]]
    pos4, off, Ls = concat(systems)
    # splice an empty system between 2 and 3
    off = np.insert(off, 3, off[3])
    Ls = np.insert(Ls, 3, np.float32(20.0))
    import torch

    from paper_1901_08088_gb300 import NeighborList

    nl = NeighborList(0)
    nl.build_batched(torch.from_numpy(pos4).cuda(), off, Ls)
    nl.query(2.8)
    rows, counts = nl.neighbors()
    rows, counts = rows.cpu().numpy(), counts.cpu().numpy()
    real = [0, 1, 2, 4, 5, 6]
    for k, s in zip(real, systems):
        a, b = off[k], off[k + 1]
        ro, co = oracle_list(s, method="brute")
        assert_same_lists(rows[a:b] - a, counts[a:b], ro, co)
    nl.close()


@pytest.mark.parametrize("traversal,wp", [(0, 32), (1, 32), (1, 8), (1, 4), (1, 1)])
def test_two_type_batched_systems(traversal, wp):
    systems = workloads.two_type_lj(seed=8, n_sys=3, n=5000)
    rows, counts, off, nl = _batched(systems, n_types=2, traversal=traversal, wp=wp)
    _check_systems(systems, rows, counts, off)
    nl.close()


@pytest.mark.slow
def test_full_ensemble_256():
    systems = workloads.workload("ensemble_256", seed=0)
    rows, counts, off, nl = _batched(systems)
    _check_systems(systems, rows, counts, off)
    nl.close()
