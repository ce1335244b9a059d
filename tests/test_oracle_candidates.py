"""Pins for the oracle's candidate lists (Alg. 1 without the exact leaf
filter, Sec. 2.3; CPU only).

The candidate list is pinned against an FP64 restatement written here with
numpy.  Both overlap tests in the oracle round their distances toward zero,
so they can only shrink them: every image whose padded sphere reaches the
root box, and every leaf box it reaches under that image, in exact FP64
arithmetic, must be listed (completeness), and every listed entry must be
within the padded radius up to FP32 rounding (soundness).  The candidates
also contain the exact list, grow with the radius, and repeat an index once
per image that lists it.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads


def _padded_r2(r, L):
    """Padded radius of reading c3 in exact arithmetic, rounded up to FP32,
    and its square rounded up: r (1 + 2^-20) + 2^-19 L."""
    def up(x):
        f = np.float32(float(x))
        if Fraction(float(f)) < x:
            f = np.nextafter(f, np.float32(np.inf))
        return f

    exact = Fraction(float(np.float32(r))) * (1 + Fraction(1, 2 ** 20)) + Fraction(float(np.float32(L))) / 2 ** 19
    rs = up(exact)
    # the reading forms the sum in FP64 first: at most one FP64 rounding away
    assert abs(Fraction(float(rs)) - exact) <= Fraction(float(rs)) * Fraction(1, 2 ** 22)
    return float(up(Fraction(float(rs)) ** 2))


def _boxes(pos, types, n_types, L, leaf_bits=10):
    tree = oracle.lbvh_build(pos, types, np.full(n_types, np.float32(L), np.float32))
    lo = np.zeros((len(pos), 3), np.float64)
    hi = np.zeros((len(pos), 3), np.float64)
    for j, p in enumerate(pos):
        if leaf_bits == 0:   # FP32 leaves: the point itself
            lo[j] = hi[j] = p
            continue
        fr = tree["frame"][types[j]]
        h = fr[3:] if leaf_bits == 10 else oracle.frame_width(tree["root"][types[j], :3],
                                                              tree["root"][types[j], 3:], leaf_bits)
        ql, qh = oracle.quantize_box(p, p, fr[:3], h, bits=leaf_bits)
        a, b = oracle.dequantize(ql, qh, fr[:3], h)
        lo[j], hi[j] = a, b
    return tree["root"].astype(np.float64), lo, hi


def _box_d2(p, lo, hi):
    g = np.maximum(np.maximum(lo - p, p - hi), 0.0)
    return (g * g).sum(-1)


def _expected(pos, types, n_types, L, rl, leaf_bits=10):
    """FP64 restatement: per (i, j) the images that certainly list j (all
    distances within rs2) and the images that may list it (within rs2 up to a
    relative 1e-6)."""
    root, lo, hi = _boxes(pos, types, n_types, L, leaf_bits)
    n = len(pos)
    L32 = np.float32(L)
    must = np.zeros((n, n), np.int32)
    may = np.zeros((n, n), np.int32)
    for i in range(n):
        a = types[i]
        for b in range(n_types):
            r = rl[a, b]
            if not r > 0 or not (types == b).any():
                continue
            rs2 = _padded_r2(r, L)
            for m in range(27):
                sh = np.array([m // 9 - 1, (m // 3) % 3 - 1, m % 3 - 1])
                p = np.array([pos[i, d] if sh[d] == 0 else np.float32(pos[i, d] + sh[d] * L32)
                              for d in range(3)], np.float64)
                rd2 = _box_d2(p, root[b, :3], root[b, 3:])
                if rd2 > rs2 * (1 + 1e-6):
                    continue
                d2 = _box_d2(p[None, :], lo, hi)
                sel = types == b
                sel[i] = False
                may[i] += (sel & (d2 <= rs2 * (1 + 1e-6))).astype(np.int32)
                if rd2 <= rs2:
                    must[i] += (sel & (d2 <= rs2)).astype(np.int32)
    return must, may


def _multiplicity(rows, counts, n):
    mult = np.zeros((n, n), np.int32)
    for i in range(n):
        for j in rows[i, : counts[i]]:
            mult[i, j] += 1
    return mult


@pytest.mark.parametrize("leaf_bits", [10, 21, 0])
@pytest.mark.parametrize("n,L,r,n_types,seed", [(1500, 15.0, 2.5, 1, 1), (1200, 12.0, 2.0, 2, 2),
                                                (300, 9.0, 4.4, 1, 3)])
def test_candidates_between_fp64_bounds(n, L, r, n_types, seed, leaf_bits):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, L, size=(n, 3)).astype(np.float32)
    pos[pos >= np.float32(L)] = 0
    types = rng.integers(0, n_types, n).astype(np.int32)
    rl = np.full((n_types, n_types), r, np.float32)
    if n_types == 2:
        rl = np.array([[r, r * 1.3], [r * 1.3, r * 0.7]], np.float32)
    rows, counts = oracle.candidates(pos, L, rl, types, n_types, cap=2048, leaf_bits=leaf_bits)
    assert counts.max() <= 2048
    mult = _multiplicity(rows, counts, n)
    must, may = _expected(pos, types, n_types, L, rl, leaf_bits)
    assert (mult >= must).all(), np.argwhere(mult < must)[:5]
    assert (mult <= may).all(), np.argwhere(mult > may)[:5]


def test_candidates_contain_exact_list_and_few_false_positives():
    s = workloads.workload("lj_n4096_rho0.6", seed=0)
    rc, cc = oracle.candidates(s.pos, s.L, s.r_list)
    ro, co = oracle.nlist(s.pos, s.L, s.r_list, method="brute")
    cand = oracle.rows_as_sets(rc, cc)
    exact = oracle.rows_as_sets(ro, co)
    assert all(exact[i] <= cand[i] for i in range(s.n))
    fp = (cc - co).mean()
    # 10-bit leaf boxes (bin width L/1023) and the radius padding add a few
    # percent at most (Sec. 4.1 reports about 5% at its state points)
    assert 0 < fp < 0.05 * co.mean()


def test_candidates_grow_with_the_radius_and_respect_zero_radii():
    rng = np.random.default_rng(4)
    n, L = 2000, 16.0
    pos = rng.uniform(0, L, size=(n, 3)).astype(np.float32)
    types = rng.integers(0, 2, n).astype(np.int32)
    small = np.array([[2.0, 1.5], [1.5, 0.0]], np.float32)
    big = np.array([[2.5, 2.0], [2.0, 1.0]], np.float32)
    rs_, cs = oracle.candidates(pos, L, small, types, 2)
    rb, cb = oracle.candidates(pos, L, big, types, 2)
    a = oracle.rows_as_sets(rs_, cs)
    b = oracle.rows_as_sets(rb, cb)
    assert all(a[i] <= b[i] for i in range(n))
    for i in np.nonzero(types == 1)[0][:200]:
        assert all(types[j] == 0 for j in a[i])   # r[1][1] = 0: no type-1 entries


def test_candidates_segregated_types_use_each_trees_root_box():
    # type 1 only in x < L/3, type 0 only above: the two trees' root boxes
    # differ, and type-0 particles near x = L reach type 1 only through the
    # image across the x = 0 face
    rng = np.random.default_rng(5)
    n, L = 1200, 14.0
    types = (np.arange(n) % 3 == 0).astype(np.int32)
    pos = rng.uniform(0, L, size=(n, 3)).astype(np.float32)
    pos[:, 0] = np.where(types == 1, rng.uniform(0, L / 3, n), rng.uniform(L / 3, L, n)).astype(np.float32)
    pos[pos >= np.float32(L)] = 0
    rl = np.array([[2.2, 2.6], [2.6, 1.8]], np.float32)
    rows, counts = oracle.candidates(pos, L, rl, types, 2, cap=1024)
    mult = _multiplicity(rows, counts, n)
    must, may = _expected(pos, types, 2, L, rl)
    assert must.sum() > 0
    assert (mult >= must).all(), np.argwhere(mult < must)[:5]
    assert (mult <= may).all(), np.argwhere(mult > may)[:5]


def test_false_positives_shrink_with_the_leaf_precision():
    # a leaf box contains its point, and the overlap test is monotone in the
    # box: FP32-point candidates are a subset of the 21-bit ones and of the
    # 10-bit ones; the 21-bit boxes (bin width L / 2^21) leave almost no false
    # positives beyond the radius padding, the 10-bit ones a few percent
    s = workloads.workload("lj_n4096_rho0.6", seed=0)
    ro, co = oracle.nlist(s.pos, s.L, s.r_list, method="brute")
    out = {}
    for bits in (0, 21, 10):
        rc, cc = oracle.candidates(s.pos, s.L, s.r_list, cap=512, leaf_bits=bits)
        out[bits] = (oracle.rows_as_sets(rc, cc), cc)
    for i in range(s.n):
        assert out[0][0][i] <= out[21][0][i] and out[0][0][i] <= out[10][0][i]
    fp = {b: (out[b][1] - co).mean() for b in out}
    assert 0 <= fp[0] <= fp[21] < fp[10]
    assert fp[21] < 0.002 * co.mean() and fp[10] < 0.05 * co.mean()
