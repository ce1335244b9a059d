"""The allocation-free LJ entry point, through the C ABI.

qbvh_lj_forward_noalloc serves callers that cannot allocate device memory when
they need forces (a locked allocator, a plugin whose host owns every
allocation, a loop where cudaMalloc/cudaFree are not allowed).  It keeps its
per-block sums and its error word in a fixed variable inside the library
instead of allocating.  Checked here against the regular entry point (two
calls in a row: the shared variable carries nothing over), against the FP64
oracle on systems larger than one sweep of its fixed grid (1216 blocks x 32
particles = 38,912) and with three and four types, and for its error reports.
This file is collected last so that a stop-at-first-failure run has already run
everything else; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle
import workloads
from helpers import gpu_list, oracle_list

pytestmark = pytest.mark.gpu
TOL = 1e-5
ONE_SWEEP = 1216 * 32   # particles one pass of the fixed grid covers


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _outputs(n, T):
    import torch

    return (torch.empty(n, dtype=torch.float32, device="cuda"),
            torch.empty(1, dtype=torch.float64, device="cuda"),
            torch.empty((n, 3), dtype=torch.float32, device="cuda"),
            torch.empty((1, T, T), dtype=torch.float64, device="cuda"),
            torch.empty((1, T, T), dtype=torch.float64, device="cuda"))


def _noalloc(pos4, L, T, rows, counts, E, S, rc):
    import torch

    from paper_1901_08088_gb300.qbvh import check, qbvh_lj_forward_noalloc

    out = _outputs(int(pos4.shape[0]), T)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    check(qbvh_lj_forward_noalloc(pos4, L, T, rows, counts, E, S, rc, *out, status), "noalloc")
    torch.cuda.synchronize()
    return out, int(status.item())


def _params(T, seed):
    """Symmetric per-pair eps in [0.5, 1.5] and sigma in [0.8, 1.0]."""
    rng = np.random.default_rng(seed)
    E = rng.uniform(0.5, 1.5, (T, T))
    S = rng.uniform(0.8, 1.0, (T, T))
    return np.triu(E) + np.triu(E, 1).T, np.triu(S) + np.triu(S, 1).T


def _typed_lattice(n, T, seed):
    s = workloads.jittered_lattice(n, 0.8, 0.3, seed=seed, r_cut=2.5, skin=0.3)
    s.types = np.random.default_rng(seed + 100).integers(0, T, n).astype(np.int32)
    s.n_types = T
    s.r_list = np.full((T, T), np.float32(2.5) + np.float32(0.3), np.float32)
    s.r_cut = np.full((T, T), 2.5, np.float32)
    return s


@pytest.mark.parametrize("two_types", [False, True])
def test_noalloc_matches_regular_entry_point_twice(two_types):
    import torch

    from paper_1901_08088_gb300.qbvh import check, qbvh_lj_forward

    if two_types:
        s = workloads.two_type_lj(seed=3, n_sys=1, n=6000)[0]
        E = torch.tensor(s.meta["eps"], dtype=torch.float32, device="cuda")
        S = torch.tensor(s.meta["sig"], dtype=torch.float32, device="cuda")
        rc = np.full((2, 2), 2.5, np.float32)
    else:
        s = workloads.workload("lj_n4096_rho0.6", seed=2)
        E = torch.ones((1, 1), dtype=torch.float32, device="cuda")
        S = torch.ones((1, 1), dtype=torch.float32, device="cuda")
        rc = np.full((1, 1), 3.0, np.float32)
    T = s.n_types
    _, _, nl, pos4 = gpu_list(s)
    rows, counts = nl.neighbors()
    ref = _outputs(s.n, T)
    check(qbvh_lj_forward(nl.h, pos4, E, S, rc, *ref), "qbvh_lj_forward")
    for _ in range(2):   # two calls in a row: the shared variable carries nothing over
        got, status = _noalloc(pos4, s.L, T, rows, counts, E, S, rc)
        assert status == 0
        assert abs(got[1].item() - ref[1].item()) <= TOL * abs(ref[1].item())
        assert _rel(got[0].cpu(), ref[0].cpu()) <= TOL
        assert _rel(got[2].cpu(), ref[2].cpu()) <= TOL
        for k in (3, 4):
            a, b = got[k].cpu().numpy(), ref[k].cpu().numpy()
            assert np.all(np.abs(a - b) <= TOL * np.abs(b)), (k, a, b)
    nl.close()


@pytest.mark.parametrize("n,T", [(65_536, 2), (50_000, 3), (45_000, 4)])
def test_noalloc_beyond_one_grid_sweep_against_fp64_oracle(n, T):
    """Systems larger than one sweep of the fixed grid, so that the
    grid-stride loop runs twice: energy, forces and every eps/sigma gradient
    within 1e-5 of the FP64 oracle on the oracle's own list, and the same as
    the regular entry point, on two calls in a row."""
    import torch

    from paper_1901_08088_gb300.qbvh import check, qbvh_lj_forward

    assert n > ONE_SWEEP
    s = workloads.two_type_lj(seed=5, n_sys=1, n=n)[0] if T == 2 else _typed_lattice(n, T, seed=7 + T)
    Eh, Sh = (s.meta["eps"], s.meta["sig"]) if T == 2 else _params(T, seed=T)
    E = torch.tensor(Eh, dtype=torch.float32, device="cuda")
    S = torch.tensor(Sh, dtype=torch.float32, device="cuda")
    rc = np.full((T, T), 2.5, np.float32)
    _, _, nl, pos4 = gpu_list(s)
    rows, counts = nl.neighbors()
    ro, co = oracle_list(s)
    ref64 = oracle.lj_fp64(s.pos, s.types, s.L, Eh, Sh, np.float32(2.5), ro, co)
    reg = _outputs(s.n, T)
    check(qbvh_lj_forward(nl.h, pos4, E, S, rc, *reg), "qbvh_lj_forward")
    for _ in range(2):
        got, status = _noalloc(pos4, s.L, T, rows, counts, E, S, rc)
        assert status == 0
        assert abs(got[1].item() - ref64["U"]) <= TOL * abs(ref64["U"])
        assert _rel(got[0].cpu().numpy(), ref64["e"]) <= TOL
        assert _rel(got[2].cpu().numpy(), ref64["F"]) <= TOL
        dE, dS = got[3].cpu().numpy()[0], got[4].cpu().numpy()[0]
        assert np.all(np.abs(dE - ref64["dE"]) <= TOL * np.abs(ref64["dE"])), (dE, ref64["dE"])
        assert np.all(np.abs(dS - ref64["dS"]) <= TOL * np.abs(ref64["dS"])), (dS, ref64["dS"])
        # the regular entry point on the same list
        assert abs(got[1].item() - reg[1].item()) <= TOL * abs(reg[1].item())
        assert _rel(got[2].cpu(), reg[2].cpu()) <= TOL
    nl.close()


def test_noalloc_reports_bad_types_and_indices():
    """A type outside [0, n_types) is reported (BAD_TYPE), not clamped: that
    particle and its pairs are left out and the energy is NaN.  A row entry
    outside [0, n) is reported as INTERNAL.  A clean call afterwards reports
    OK again (the error word is cleared by every call)."""
    import torch

    from paper_1901_08088_gb300 import _lib

    s = workloads.two_type_lj(seed=8, n_sys=1, n=3000)[0]
    E = torch.tensor(s.meta["eps"], dtype=torch.float32, device="cuda")
    S = torch.tensor(s.meta["sig"], dtype=torch.float32, device="cuda")
    rc = np.full((2, 2), 2.5, np.float32)
    _, _, nl, pos4 = gpu_list(s)
    rows, counts = nl.neighbors()
    bad = pos4.clone()
    bad[17, 3] = torch.tensor([2], dtype=torch.int32).view(torch.float32)[0]   # type 2 of 2
    out, status = _noalloc(bad, s.L, 2, rows, counts, E, S, rc)
    assert status == _lib.QBVH_ERR_BAD_TYPE
    assert np.isnan(out[1].item())
    assert float(out[2][17].abs().sum()) == 0.0 and float(out[0][17]) == 0.0
    bad[17, 3] = torch.tensor([-1], dtype=torch.int32).view(torch.float32)[0]
    _, status = _noalloc(bad, s.L, 2, rows, counts, E, S, rc)
    assert status == _lib.QBVH_ERR_BAD_TYPE
    rows_bad = rows.clone()
    rows_bad[5, 0] = s.n
    out, status = _noalloc(pos4, s.L, 2, rows_bad, counts, E, S, rc)
    assert status == _lib.QBVH_ERR_INTERNAL and np.isnan(out[1].item())
    out, status = _noalloc(pos4, s.L, 2, rows, counts, E, S, rc)
    assert status == _lib.QBVH_OK and np.isfinite(out[1].item())
    nl.close()


def test_noalloc_rejects_type_counts_beyond_its_fixed_array():
    import torch

    from paper_1901_08088_gb300 import _lib
    from paper_1901_08088_gb300.qbvh import qbvh_lj_forward_noalloc

    n = 64
    pos4 = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    rows = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    E = torch.ones((5, 5), dtype=torch.float32, device="cuda")
    U = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    rc = np.ones((5, 5), np.float32)
    rc_code = qbvh_lj_forward_noalloc(pos4, 10.0, 5, rows, counts, E, E, rc, None, U, None, None, None, st)
    assert rc_code == _lib.QBVH_ERR_INVALID_ARG
    # the status output is required
    E1 = torch.ones((1, 1), dtype=torch.float32, device="cuda")
    rc_code = qbvh_lj_forward_noalloc(pos4, 10.0, 1, rows, counts, E1, E1, np.ones((1, 1), np.float32), None, U,
                                      None, None, None, None)
    assert rc_code == _lib.QBVH_ERR_INVALID_ARG
