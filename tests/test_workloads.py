"""Generator checks (CPU): the seeded inputs have the shapes the workloads ask for."""
import numpy as np
import pytest

import workloads


def test_jittered_lattice_shape_and_domain():
    s = workloads.jittered_lattice(4096, 0.6, 0.3, seed=0, r_cut=3.0, skin=0.4)
    assert s.pos.dtype == np.float32 and s.pos.shape == (4096, 3)
    assert (s.pos >= 0).all() and (s.pos < s.L).all()
    assert s.L == np.float32((4096 / 0.6) ** (1 / 3))
    assert s.r_list[0, 0] == np.float32(3.4)
    again = workloads.jittered_lattice(4096, 0.6, 0.3, seed=0, r_cut=3.0, skin=0.4)
    assert np.array_equal(s.pos, again.pos)


def test_non_cube_counts_pick_distinct_sites():
    s = workloads.jittered_lattice(1000 + 7, 0.5, 0.0, seed=2)
    # zero jitter: the occupied sites are distinct lattice points
    assert np.unique(s.pos, axis=0).shape[0] == s.n


@pytest.mark.slow
def test_binary_mixture_constraints():
    s = workloads.binary_mixture(seed=0, n_small=20000)
    big = s.pos[s.types == 1].astype(np.float64)
    small = s.pos[s.types == 0].astype(np.float64)
    assert big.shape[0] == 400 and small.shape[0] == 20000
    L = float(s.L)
    for c in big[:50]:
        d = small - c
        d -= L * np.rint(d / L)
        assert (np.sqrt((d * d).sum(1)) >= 5.0 - 1e-4).all()
        e = big - c
        e -= L * np.rint(e / L)
        r = np.sqrt((e * e).sum(1))
        assert (r[r > 0] >= 10.0 - 1e-4).all()
    assert s.r_list[0, 1] == np.float32(5.9) and s.r_list[1, 1] == np.float32(10.4)


def test_default_mixture_small_count():
    free = 100.0 ** 3 - 400 * 4.0 / 3.0 * np.pi * 125.0
    assert int(round(0.5 * free)) == 395280


def test_ensemble_and_two_type():
    ens = workloads.batched_ensemble(seed=1, n_sys=8)
    assert all(500 <= s.n <= 50000 for s in ens)
    assert all(float(s.L) / 2 > 2.8 for s in ens)
    tt = workloads.two_type_lj(seed=0, n_sys=2, n=4096)
    assert tt[0].types.sum() == 2048 and tt[0].n_types == 2


def test_pack_float4_roundtrip():
    s = workloads.jittered_lattice(64, 0.5, 0.1, seed=1)
    t = np.arange(64, dtype=np.int32) % 3
    p4 = workloads.pack_float4(s.pos, t)
    assert np.array_equal(p4[:, :3], s.pos) and np.array_equal(p4.view(np.int32)[:, 3], t)


def test_spinodal_like_is_inhomogeneous_and_exact_in_n():
    # a small version of the liquid/vapor stand-in (Sec. 4.3): exact N, inside
    # the box, liquid mass fraction from the lever rule, and local densities
    # spanning vapor to liquid
    s = workloads.spinodal_like(60_000, 0.2, seed=1, wavelength=10.0)
    assert s.n == 60_000 and s.pos.dtype == np.float32
    assert (s.pos >= 0).all() and (s.pos < s.L).all()
    frac_liquid = s.meta["n_liquid"] / s.n
    assert abs(frac_liquid - 0.72 * (0.18 / 0.70) / 0.2) < 0.05
    nc = 16   # cells of ~4 sigma resolve domains of wavelength 10
    h, _ = np.histogramdd(s.pos, bins=nc, range=[(0, float(s.L))] * 3)
    d = h.ravel() / (float(s.L) / nc) ** 3
    assert np.percentile(d, 10) < 0.05 and np.percentile(d, 90) > 0.4
    s64 = workloads.spinodal_like(60_000, 0.2, seed=1, wavelength=10.0, double=True)
    assert s64.pos.dtype == np.float64 and (s64.pos < s64.L).all() and s64.n == 60_000
