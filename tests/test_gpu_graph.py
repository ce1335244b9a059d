"""Batched build + query replayed from a CUDA graph: every replay equals the
oracle for the positions currently in the input buffer, overflow triggers a
recapture with a larger capacity, and the per-system loop gives the same lists."""
import numpy as np
import pytest

import workloads
from helpers import assert_same_lists, concat, oracle_list

pytestmark = pytest.mark.gpu


def _check(systems, rows, counts, off):
    for k, s in enumerate(systems):
        a, b = off[k], off[k + 1]
        ro, co = oracle_list(s, method="brute" if s.n < 3000 else "cell")
        assert_same_lists(rows[a:b] - a, counts[a:b], ro, co)


def test_graph_replay_tracks_buffer_updates():
    import torch

    from paper_1901_08088_gb300 import BatchedNeighborList

    systems = workloads.batched_ensemble(seed=21, n_sys=10, n_min=300, n_max=4000)
    pos4, off, Ls = concat(systems)
    buf = torch.from_numpy(pos4).cuda()
    b = BatchedNeighborList(buf, off, Ls, systems[0].r_list, cap=64)
    assert b.run() == 0
    rows, counts = b.neighbors()
    _check(systems, rows.cpu().numpy(), counts.cpu().numpy(), off)
    # move every particle (wrapped) and replay the same graph
    moved = []
    rng = np.random.default_rng(3)
    for s in systems:
        p = np.mod(s.pos.astype(np.float64) + rng.uniform(-0.2, 0.2, s.pos.shape), float(s.L)).astype(np.float32)
        p[p >= s.L] = 0
        moved.append(workloads.System(pos=p, types=s.types, L=s.L, n_types=1, r_list=s.r_list, r_cut=s.r_cut))
    p4, _, _ = concat(moved)
    buf.copy_(torch.from_numpy(p4).cuda())
    captures = b.captures
    assert b.run() == 0
    rows, counts = b.neighbors()
    _check(moved, rows.cpu().numpy(), counts.cpu().numpy(), off)
    assert b.captures >= captures
    b.close()


def test_graph_recaptures_when_rows_overflow():
    import torch

    from paper_1901_08088_gb300 import BatchedNeighborList

    systems = workloads.batched_ensemble(seed=22, n_sys=6, n_min=500, n_max=3000)
    pos4, off, Ls = concat(systems)
    b = BatchedNeighborList(torch.from_numpy(pos4).cuda(), off, Ls, systems[0].r_list, cap=4)
    assert b.run() == 0
    assert b.cap >= 32 and b.captures >= 1
    rows, counts = b.neighbors()
    _check(systems, rows.cpu().numpy(), counts.cpu().numpy(), off)
    b.close()


def test_per_system_loop_equals_batched():
    import torch

    from paper_1901_08088_gb300 import BatchedNeighborList, PerSystemLoop

    systems = workloads.batched_ensemble(seed=23, n_sys=8, n_min=300, n_max=3000)
    pos4, off, Ls = concat(systems)
    buf = torch.from_numpy(pos4).cuda()
    b = BatchedNeighborList(buf, off, Ls, systems[0].r_list, cap=128)
    assert b.run() == 0
    rows, counts = b.neighbors()
    rows, counts = rows.cpu().numpy(), counts.cpu().numpy()
    loop = PerSystemLoop(buf, off, Ls, systems[0].r_list, cap=128)
    assert loop.run() == 0
    for k, nl in enumerate(loop.handles):
        r, c = nl.neighbors()
        a, e = off[k], off[k + 1]
        assert_same_lists(rows[a:e] - a, counts[a:e], r.cpu().numpy(), c.cpu().numpy())
    loop.close()
    b.close()


def test_autotuner_returns_a_valid_choice():
    import torch

    from paper_1901_08088_gb300 import NeighborList, autotune, _lib

    s = workloads.workload("lj_n4096_rho0.6", seed=4)
    pos4 = torch.from_numpy(workloads.pack_float4(s.pos, s.types)).cuda()
    nl = NeighborList(0)

    def step(opts):
        for k, v in opts.items():
            nl.set_option(k, v)
        nl.build(pos4, s.L)
        nl.query_async(s.r_list, 256)

    best, ms, log = autotune.tune(step, reps=2, warmup=1, sweeps=1)
    assert ms > 0 and len(log) > 1
    valid = {**autotune.OPTION_SPACE, **autotune.OPTIONAL_SPACE}
    for k, v in best.items():
        assert v in valid[k]
    # the chosen options still give the exact list
    step(best)
    torch.cuda.synchronize()
    assert nl.query_status()[0] == _lib.QBVH_OK
    rows, counts = nl.neighbors()
    ro, co = oracle_list(s, method="brute")
    assert_same_lists(rows.cpu().numpy(), counts.cpu().numpy(), ro, co)
    nl.close()
