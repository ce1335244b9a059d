"""Failure detection without a GPU fault: a bounded device wait that is made to
run out reports an error and leaves the context usable; host-side fault
injection (QBVH_FAULT) drives the OOM, timeout and overflow paths."""
import os

import numpy as np
import pytest

import workloads
from helpers import assert_same_lists, gpu_list, oracle_list

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    from paper_1901_08088_gb300 import _lib
    from paper_1901_08088_gb300.qbvh import qbvh_selftest_wait_timeout

    assert qbvh_selftest_wait_timeout(0) == _lib.QBVH_ERR_DEVICE_TIMEOUT
    # the same process keeps working
    s = workloads.workload("lj_n4096_rho0.6", seed=5)
    rg, cg, nl, _ = gpu_list(s)
    ro, co = oracle_list(s, method="brute")
    assert_same_lists(rg, cg, ro, co)
    nl.close()


@pytest.mark.parametrize("fault,expect", [("timeout", "QBVH_ERR_DEVICE_TIMEOUT"), ("overflow", "QBVH_ERR_OVERFLOW"),
                                          ("alloc", "QBVH_ERR_OOM")])
def test_host_fault_injection(fault, expect):
    import torch

    from paper_1901_08088_gb300 import NeighborList, _lib
    from paper_1901_08088_gb300.qbvh import qbvh_build

    s = workloads.workload("lj_n4096_rho0.6", seed=6)
    pos4 = torch.from_numpy(workloads.pack_float4(s.pos, s.types)).cuda()
    old = os.environ.get("QBVH_FAULT")
    os.environ["QBVH_FAULT"] = fault
    try:
        nl = NeighborList(0)      # the handle reads QBVH_FAULT when it is created
    finally:
        if old is None:
            del os.environ["QBVH_FAULT"]
        else:
            os.environ["QBVH_FAULT"] = old
    code = getattr(_lib, expect)
    if fault == "alloc":
        assert qbvh_build(nl.h, pos4, s.L) == code
    else:
        nl.build(pos4, s.L)
        assert nl.query(s.r_list, raise_on_error=False) == code
    nl.close()
    # a handle created afterwards is unaffected
    rg, cg, nl2, _ = gpu_list(s)
    ro, co = oracle_list(s, method="brute")
    assert_same_lists(rg, cg, ro, co)
    nl2.close()
