"""GPU parity of the fused Lennard-Jones pass (Eq. 1, truncated and shifted)
against the FP64 oracle: energy, forces and eps/sigma gradients within 1e-5
relative, through the autograd wrapper and the C ABI."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import concat, gpu_list, oracle_list

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _run(nl, s, pos4, E, S, rc, weights=None):
    import torch

    from paper_1901_08088_gb300 import lj_energy

    xyz = torch.from_numpy(s.pos).cuda().requires_grad_(True)
    eps = torch.tensor(E, dtype=torch.float32, device="cuda", requires_grad=True)
    sig = torch.tensor(S, dtype=torch.float32, device="cuda", requires_grad=True)
    U = lj_energy(nl, xyz, eps, sig, rc, pos4=pos4)
    w = torch.ones_like(U) if weights is None else torch.tensor(weights, dtype=torch.float64, device="cuda")
    (U * w).sum().backward()
    return U.detach().cpu().numpy(), xyz.grad.cpu().numpy(), eps.grad.cpu().numpy(), sig.grad.cpu().numpy()


@pytest.mark.parametrize("zorder", [0, 1])
@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_single_type_energy_forces(lanes, zorder):
    from paper_1901_08088_gb300 import _lib

    s = workloads.workload("lj_n4096_rho0.6", seed=1)
    rg, cg, nl, pos4 = gpu_list(s)
    nl.set_option(_lib.QBVH_OPT_LJ_LANES, lanes)
    nl.set_option(_lib.QBVH_OPT_LJ_ZORDER, zorder)
    U, gx, ge, gs = _run(nl, s, pos4, [[1.0]], [[1.0]], 3.0)
    ro, co = oracle_list(s, method="brute")
    ref = oracle.lj_fp64(s.pos, s.types, s.L, [[1.0]], [[1.0]], np.float32(3.0), ro, co)
    assert abs(U[0] - ref["U"]) <= TOL * abs(ref["U"])
    assert _rel(-gx, ref["F"]) <= TOL
    assert abs(ge[0, 0] - ref["dE"][0, 0]) <= TOL * abs(ref["dE"][0, 0])
    assert abs(gs[0, 0] - ref["dS"][0, 0]) <= TOL * abs(ref["dS"][0, 0])
    nl.close()


@pytest.mark.parametrize("lanes", [1, 8, 32])
def test_two_types_parameter_gradients_and_weighted_backward(lanes):
    from paper_1901_08088_gb300 import _lib

    sys0 = workloads.two_type_lj(seed=2, n_sys=1, n=8000)[0]
    E, S = sys0.meta["eps"], sys0.meta["sig"]
    rg, cg, nl, pos4 = gpu_list(sys0)
    nl.set_option(_lib.QBVH_OPT_LJ_LANES, lanes)
    U, gx, ge, gs = _run(nl, sys0, pos4, E, S, 2.5, weights=[-0.75])
    ro, co = oracle_list(sys0)
    ref = oracle.lj_fp64(sys0.pos, sys0.types, sys0.L, E, S, np.float32(2.5), ro, co)
    assert abs(U[0] - ref["U"]) <= TOL * abs(ref["U"])
    assert _rel(-gx / -0.75, ref["F"]) <= TOL
    for a in range(2):
        for b in range(2):
            assert abs(ge[a, b] / -0.75 - ref["dE"][a, b]) <= TOL * abs(ref["dE"][a, b]), (a, b)
            assert abs(gs[a, b] / -0.75 - ref["dS"][a, b]) <= TOL * abs(ref["dS"][a, b]), (a, b)
    nl.close()


def test_energy_uses_r_cut_not_r_list():
    s = workloads.workload("lj_n4096_rho0.6", seed=3)
    rg, cg, nl, pos4 = gpu_list(s)     # r_list = 3.4
    U, gx, _, _ = _run(nl, s, pos4, [[1.0]], [[1.0]], 2.5)
    ro, co = oracle_list(s, method="brute")
    ref = oracle.lj_fp64(s.pos, s.types, s.L, [[1.0]], [[1.0]], np.float32(2.5), ro, co)
    assert abs(U[0] - ref["U"]) <= TOL * abs(ref["U"])
    assert _rel(-gx, ref["F"]) <= TOL
    nl.close()


def test_batched_two_type_systems():
    import torch

    from paper_1901_08088_gb300 import NeighborList

    systems = workloads.two_type_lj(seed=4, n_sys=4, n=8192)
    E, S = systems[0].meta["eps"], systems[0].meta["sig"]
    pos4, off, Ls = concat(systems)
    nl = NeighborList(0)
    p4 = torch.from_numpy(pos4).cuda()
    nl.build_batched(p4, off, Ls, n_types=2)
    nl.query(2.8)
    allpos = np.concatenate([s.pos for s in systems])
    big = workloads.System(pos=allpos, types=np.concatenate([s.types for s in systems]), L=Ls[0],
                           n_types=2, r_list=systems[0].r_list, r_cut=systems[0].r_cut)
    U, gx, ge, gs = _run(nl, big, p4, E, S, 2.5, weights=[1.0, 2.0, -1.0, 0.5])
    w = np.array([1.0, 2.0, -1.0, 0.5])
    dE = np.zeros((2, 2))
    dS = np.zeros((2, 2))
    for k, s in enumerate(systems):
        a, b = off[k], off[k + 1]
        ro, co = oracle_list(s)
        ref = oracle.lj_fp64(s.pos, s.types, s.L, E, S, np.float32(2.5), ro, co)
        assert abs(U[k] - ref["U"]) <= TOL * abs(ref["U"])
        assert _rel(-gx[a:b] / w[k], ref["F"]) <= TOL
        dE += w[k] * ref["dE"]
        dS += w[k] * ref["dS"]
    assert np.all(np.abs(ge - dE) <= TOL * np.abs(dE))
    assert np.all(np.abs(gs - dS) <= TOL * np.abs(dS))
    nl.close()


@pytest.mark.slow
def test_config2_full_size_energy_forces():
    s = workloads.workload("lj_n2097152_rho0.8", seed=0)
    rg, cg, nl, pos4 = gpu_list(s)
    U, gx, ge, gs = _run(nl, s, pos4, [[1.0]], [[1.0]], 3.0)
    ro, co = oracle_list(s)
    ref = oracle.lj_fp64(s.pos, s.types, s.L, [[1.0]], [[1.0]], np.float32(3.0), ro, co)
    assert abs(U[0] - ref["U"]) <= TOL * abs(ref["U"])
    assert _rel(-gx, ref["F"]) <= TOL
    nl.close()


@pytest.mark.slow
def test_config5_full_two_type_batched_gradients():
    """32 systems x 65,536 particles, two types, per-pair eps/sigma: energies,
    forces and eps/sigma gradients of every system within 1e-5 of FP64."""
    import torch

    from paper_1901_08088_gb300 import NeighborList

    systems = workloads.workload("lj2type_32x65536", seed=0)
    E, S = systems[0].meta["eps"], systems[0].meta["sig"]
    pos4, off, Ls = concat(systems)
    nl = NeighborList(0)
    p4 = torch.from_numpy(pos4).cuda()
    nl.build_batched(p4, off, Ls, n_types=2)
    nl.query(2.8)
    allpos = np.concatenate([s.pos for s in systems])
    big = workloads.System(pos=allpos, types=np.concatenate([s.types for s in systems]), L=Ls[0],
                           n_types=2, r_list=systems[0].r_list, r_cut=systems[0].r_cut)
    rng = np.random.default_rng(1)
    w = rng.uniform(0.5, 1.5, len(systems))
    U, gx, ge, gs = _run(nl, big, p4, E, S, 2.5, weights=w.tolist())
    dE = np.zeros((2, 2))
    dS = np.zeros((2, 2))
    worst = {"U": 0.0, "F": 0.0}
    for k, s in enumerate(systems):
        a, b = off[k], off[k + 1]
        ro, co = oracle_list(s)
        ref = oracle.lj_fp64(s.pos, s.types, s.L, E, S, np.float32(2.5), ro, co)
        worst["U"] = max(worst["U"], abs(U[k] - ref["U"]) / abs(ref["U"]))
        worst["F"] = max(worst["F"], _rel(-gx[a:b] / w[k], ref["F"]))
        dE += w[k] * ref["dE"]
        dS += w[k] * ref["dS"]
    err_e = np.max(np.abs(ge - dE) / np.abs(dE))
    err_s = np.max(np.abs(gs - dS) / np.abs(dS))
    print(f"config 5 errors vs FP64: U {worst['U']:.2e}, F {worst['F']:.2e}, dU/deps {err_e:.2e}, "
          f"dU/dsigma {err_s:.2e}")
    assert worst["U"] <= TOL and worst["F"] <= TOL and err_e <= TOL and err_s <= TOL
    nl.close()
