"""Run-to-run determinism of the GPU path.

Row order is unspecified by the interface, but no step of the build or the
walk takes an order from an atomic: the sort is stable (Sec. 3.1), the
hierarchy follows the sorted keys (Sec. 2.1) and each row is written by the
warp that walks for its particle.  So a rebuild of the same input must give
the same tree words and the same rows entry for entry, and the Lennard-Jones
pass (per-block FP64 records added in a fixed order) the same bits."""
import numpy as np
import pytest

import workloads
from helpers import concat, gpu_list

pytestmark = pytest.mark.gpu


def _masked(rows, counts):
    c = np.minimum(counts, rows.shape[1])
    return np.where(np.arange(rows.shape[1])[None, :] < c[:, None], rows, -1)


@pytest.mark.parametrize("bundle", [16, 32])
@pytest.mark.parametrize("name", ["lj_n4096_rho0.6", "mixture_small"])
def test_rebuild_gives_identical_tree_and_rows(name, bundle):
    if name == "mixture_small":
        s = workloads.binary_mixture(seed=5, L=40.0, n_large=20, n_small=25000)
    else:
        s = workloads.workload(name, seed=5)
    runs = []
    for _ in range(2):
        rows, counts, nl, _ = gpu_list(s, bundle=bundle)
        t = nl.tree()
        nodes = t["nodes"].cpu().numpy().copy()
        nodes[t["seg_start"].cpu().numpy()[1:] - 1] = 0   # each tree's unused last slot
        runs.append((_masked(rows, counts), counts, nodes, t["leaves"].cpu().numpy()))
        # a second query on the same handle and build
        nl.query(s.r_list)
        r2, c2 = nl.neighbors()
        r2, c2 = r2.cpu().numpy(), c2.cpu().numpy()
        assert np.array_equal(c2, counts)
        assert np.array_equal(_masked(r2, c2), runs[-1][0])
        nl.close()
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)


def test_batched_rebuild_gives_identical_rows():
    import torch
    from paper_1901_08088_gb300 import NeighborList

    systems = workloads.batched_ensemble(seed=6, n_sys=12, n_min=200, n_max=3000)
    pos4, off, Ls = concat(systems)
    out = []
    for _ in range(2):
        nl = NeighborList(0)
        nl.build_batched(torch.from_numpy(pos4).cuda(), off, Ls)
        nl.query(systems[0].r_list)
        rows, counts = nl.neighbors()
        rows, counts = rows.cpu().numpy(), counts.cpu().numpy()
        out.append((_masked(rows, counts), counts))
        nl.close()
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][0], out[1][0])


@pytest.mark.parametrize("lanes", [1, 2, 8])
def test_lj_results_repeat_bit_for_bit(lanes):
    import torch
    from paper_1901_08088_gb300 import _lib, lj_energy

    s = workloads.two_type_lj(seed=7, n_sys=1, n=8000)[0]
    E, S = s.meta["eps"], s.meta["sig"]
    _, _, nl, pos4 = gpu_list(s)
    nl.set_option(_lib.QBVH_OPT_LJ_LANES, lanes)
    res = []
    for _ in range(3):
        xyz = torch.from_numpy(s.pos).cuda().requires_grad_(True)
        eps = torch.tensor(E, dtype=torch.float32, device="cuda", requires_grad=True)
        sig = torch.tensor(S, dtype=torch.float32, device="cuda", requires_grad=True)
        U = lj_energy(nl, xyz, eps, sig, 2.5, pos4=pos4)
        U.sum().backward()
        res.append([U.detach().cpu().numpy(), xyz.grad.cpu().numpy(), eps.grad.cpu().numpy(),
                    sig.grad.cpu().numpy()])
    for r in res[1:]:
        for a, b in zip(res[0], r):
            assert a.tobytes() == b.tobytes()
    nl.close()
