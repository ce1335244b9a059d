"""Alg. 1 as written (no exact leaf test): the candidate list is a superset of
the exact list, and its false positives per particle on the paper's LJ state
points (Sec. 4.1: N = 128,000, r_c = 3.0, rho 0.2 and 0.8; the paper reports
about 1.5 and 3.8 per particle, ~5%) are of that order on the synthetic
stand-ins.  Prints the measured counts."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import gpu_list, oracle_list

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rho", [0.2, 0.8])
def test_false_positives_per_particle(rho):
    s = workloads.jittered_lattice(128_000, rho, 0.3, seed=1, r_cut=3.0, skin=0.0)
    rg, cg, nl, _ = gpu_list(s, candidates=1, cap=512)
    ro, co = oracle_list(s, cap=512)
    sets_o = oracle.rows_as_sets(ro, co)
    for i in range(0, s.n, 257):
        assert sets_o[i] <= set(rg[i, : cg[i]].tolist())
    fp = (cg.astype(np.int64) - co).mean()
    print(f"rho {rho}: {co.mean():.2f} true neighbours, {fp:.2f} false positives per particle "
          f"({100 * fp / co.mean():.1f}%), 10-bit quantized leaves")
    assert (cg >= co).all()
    assert 0.0 < fp / co.mean() < 0.25
    nl.close()
