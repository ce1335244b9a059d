"""The allocation-free LJ entry point against the regular one.

qbvh_lj_forward_noalloc serves callers that cannot allocate device memory when
they need forces (a locked allocator, a plugin whose host owns every
allocation, a loop where cudaMalloc/cudaFree are not allowed).  It keeps its
per-block sums in a fixed array inside the library instead of allocating.
This file is collected last so that a stop-at-first-failure run has already run
everything else; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import workloads
from helpers import gpu_list

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("two_types", [False, True])
def test_noalloc_matches_regular_entry_point_twice(two_types):
    import torch

    from paper_1901_08088_gb300.qbvh import check, qbvh_lj_forward, qbvh_lj_forward_noalloc

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

    def outputs():
        return (torch.empty(s.n, dtype=torch.float32, device="cuda"),
                torch.empty(1, dtype=torch.float64, device="cuda"),
                torch.empty((s.n, 3), dtype=torch.float32, device="cuda"),
                torch.empty((1, T, T), dtype=torch.float64, device="cuda"),
                torch.empty((1, T, T), dtype=torch.float64, device="cuda"))

    ref = outputs()
    check(qbvh_lj_forward(nl.h, pos4, E, S, rc, *ref), "qbvh_lj_forward")
    for _ in range(2):   # two calls in a row: the shared array carries nothing over
        got = outputs()
        check(qbvh_lj_forward_noalloc(pos4, s.L, T, rows, counts, E, S, rc, *got), "noalloc")
        torch.cuda.synchronize()
        assert abs(got[1].item() - ref[1].item()) <= TOL * abs(ref[1].item())
        assert _rel(got[0].cpu(), ref[0].cpu()) <= TOL
        assert _rel(got[2].cpu(), ref[2].cpu()) <= TOL
        for k in (3, 4):
            a, b = got[k].cpu().numpy(), ref[k].cpu().numpy()
            assert np.all(np.abs(a - b) <= TOL * np.abs(b)), (k, a, b)
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
    rc = np.ones((5, 5), np.float32)
    rc_code = qbvh_lj_forward_noalloc(pos4, 10.0, 5, rows, counts, E, E, rc, None, U, None, None, None)
    assert rc_code == _lib.QBVH_ERR_INVALID_ARG
