"""One tree per system holding every particle type (QBVH_OPT_TYPE_TREES = 0).

With one list radius for every type pair, the list does not depend on how the
particles are split into trees: the per-type trees of Sec. 1 and Sec. 5 and
a single tree per system give the same exact list.  The single tree is the
tree of the same positions with every type set to 0, so its words are
compared with the oracle's construction of that input; the rows are compared
with the oracle's typed list.  Types are still validated, a query with
unequal radii is refused, and the LJ pass still reads each particle's type."""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads
from helpers import assert_same_lists, concat, oracle_list

pytestmark = pytest.mark.gpu


def _merged(systems, n_types, r, wp=32, f64=False):
    import torch
    from paper_1901_08088_gb300 import NeighborList, _lib

    nl = NeighborList(0)
    nl.set_option(_lib.QBVH_OPT_TYPE_TREES, 0)
    nl.set_option(_lib.QBVH_OPT_WARP_PARTICLES, wp)
    if f64:
        s = systems[0]
        nl.build_f64(torch.from_numpy(workloads.pack_double4(s.pos, s.types)).cuda(), float(s.L), n_types)
        off = np.array([0, s.n], np.int32)
    else:
        pos4, off, Ls = concat(systems)
        if len(systems) == 1:
            nl.build(torch.from_numpy(pos4).cuda(), systems[0].L, n_types)
        else:
            nl.build_batched(torch.from_numpy(pos4).cuda(), off, Ls, n_types=n_types)
    nl.query(r)
    rows, counts = nl.neighbors()
    return rows.cpu().numpy(), counts.cpu().numpy(), off, nl


@pytest.mark.parametrize("wp", [32, 8])
def test_batched_two_types_one_tree_per_system(wp):
    import torch

    systems = workloads.two_type_lj(seed=12, n_sys=4, n=6000)
    rows, counts, off, nl = _merged(systems, 2, float(systems[0].r_list[0, 0]), wp=wp)
    for k, s in enumerate(systems):
        a, b = off[k], off[k + 1]
        ro, co = oracle_list(s)
        assert_same_lists(rows[a:b] - a, counts[a:b], ro, co)
    # the tree of each system is the oracle's tree of its positions with one type
    t = {k: v.cpu() for k, v in nl.tree().items()}
    assert t["seg_start"].numel() == len(systems) + 1
    seg = np.concatenate([np.full(s.n, k, np.int32) for k, s in enumerate(systems)])
    pos = np.concatenate([s.pos for s in systems])
    Ls = np.array([s.L for s in systems], np.float32)
    o = oracle.lbvh_build(pos, seg, Ls, bundle_k=nl.get_option(1))
    assert np.array_equal(t["order"].numpy(), o["order"])
    assert np.array_equal(t["leaves"].view(torch.int32).numpy(), o["leaves"].view(np.int32))
    nodes = t["nodes"].numpy()
    for k in range(len(systems)):
        a, b = o["seg_start"][k], o["seg_start"][k + 1] - 1
        assert np.array_equal(nodes[a:b], o["nodes"][a:b])
    nl.close()


@pytest.mark.parametrize("n_types", [3, 6])
def test_single_system_several_types(n_types):
    rng = np.random.default_rng(13)
    n, L = 20000, np.float32(30.0)
    pos = rng.uniform(0, L, size=(n, 3)).astype(np.float32)
    pos[pos >= L] = 0
    types = rng.integers(0, n_types, n).astype(np.int32)
    rl = np.full((n_types, n_types), 2.7, np.float32)
    s = workloads.System(pos=pos, types=types, L=L, n_types=n_types, r_list=rl, r_cut=rl.copy())
    rows, counts, _, nl = _merged([s], n_types, rl)
    ro, co = oracle_list(s)
    assert_same_lists(rows, counts, ro, co)
    nl.close()


def test_double_precision_data_one_tree():
    s = workloads.jittered_lattice64(8000, 0.8, 0.3, seed=14, r_cut=2.5, skin=0.3)
    rng = np.random.default_rng(14)
    types = rng.integers(0, 2, s.n).astype(np.int32)
    s = dataclasses.replace(s, types=types, n_types=2, r_list=np.full((2, 2), s.r_list.flat[0], np.float32),
                            r_cut=np.full((2, 2), s.r_cut.flat[0], np.float32))
    rows, counts, _, nl = _merged([s], 2, s.r_list, f64=True)
    ro, co = oracle.nlist64(s.pos, s.L, s.r_list, s.types, 2)
    assert_same_lists(rows, counts, ro, co)
    nl.close()


def test_unequal_radii_refused_and_types_still_checked():
    import torch
    from paper_1901_08088_gb300 import NeighborList, _lib

    systems = workloads.two_type_lj(seed=15, n_sys=1, n=4000)
    s = systems[0]
    nl = NeighborList(0)
    nl.set_option(_lib.QBVH_OPT_TYPE_TREES, 0)
    assert nl.get_option(_lib.QBVH_OPT_TYPE_TREES) == 0
    pos4 = torch.from_numpy(workloads.pack_float4(s.pos, s.types)).cuda()
    nl.build(pos4, s.L, 2)
    r = np.array([[2.8, 2.8], [2.8, 2.5]], np.float32)
    assert nl.query(r, raise_on_error=False) == _lib.QBVH_ERR_INVALID_ARG
    assert nl.query(2.8, raise_on_error=False) == _lib.QBVH_OK
    bad = s.types.copy()
    bad[7] = 2   # outside [0, n_types)
    nl.build(torch.from_numpy(workloads.pack_float4(s.pos, bad)).cuda(), s.L, 2)
    assert nl.query(2.8, raise_on_error=False) == _lib.QBVH_ERR_BAD_TYPE
    nl.close()


def test_lj_reads_types_with_one_tree():
    import torch
    from paper_1901_08088_gb300 import lj_energy

    s = workloads.two_type_lj(seed=16, n_sys=1, n=8000)[0]
    E, S = s.meta["eps"], s.meta["sig"]
    rows, counts, _, nl = _merged([s], 2, float(s.r_list[0, 0]))
    pos4 = torch.from_numpy(workloads.pack_float4(s.pos, s.types)).cuda()
    xyz = torch.from_numpy(s.pos).cuda().requires_grad_(True)
    eps = torch.tensor(E, dtype=torch.float32, device="cuda", requires_grad=True)
    sig = torch.tensor(S, dtype=torch.float32, device="cuda", requires_grad=True)
    U = lj_energy(nl, xyz, eps, sig, 2.5, pos4=pos4)
    U.sum().backward()
    ro, co = oracle_list(s)
    ref = oracle.lj_fp64(s.pos, s.types, s.L, E, S, np.float32(2.5), ro, co)
    tol = 1e-5
    assert abs(U.item() - ref["U"]) <= tol * abs(ref["U"])
    gx = xyz.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(-gx - ref["F"]) <= tol * np.linalg.norm(ref["F"])
    ge, gs = eps.grad.cpu().numpy(), sig.grad.cpu().numpy()
    assert np.all(np.abs(ge - ref["dE"]) <= tol * np.abs(ref["dE"]))
    assert np.all(np.abs(gs - ref["dS"]) <= tol * np.abs(ref["dS"]))
    nl.close()
