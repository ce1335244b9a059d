"""Pins for the LBVH oracle (CPU only): Morton binning, sort, hierarchy, ropes,
fit and outward quantization (Sec. 2.1, 2.2, Fig. 3, Alg. 1 traversal).

Each oracle step is checked against something other than itself:
hand-worked Morton codes, a bit-by-bit decoder, numpy's lexsort, the radix-tree
characterisation of a node (its leaf range is exactly the keys sharing its
prefix), a stack-based pruned depth-first search (the alternative to ropes the
paper mentions in Sec. 2.1), and containment of every particle in every
ancestor's decoded quantized box.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden")
END = int(oracle.END)


def test_golden_morton_codes():
    gold = json.load(open(os.path.join(GOLD, "morton_codes.json")))
    L = np.float32(gold["L"])
    bins = np.array([c["bins"] for c in gold["cases"]], np.float64)
    pos = (bins + 0.5).astype(np.float32)
    codes = oracle.morton(pos, L)
    assert codes.tolist() == [c["code"] for c in gold["cases"]]


def _decode_bits(code):
    s = format(int(code), "030b")          # 30 bits, most significant first
    x = int(s[0::3], 2)
    y = int(s[1::3], 2)
    z = int(s[2::3], 2)
    return x, y, z


def test_morton_decodes_back_to_bins():
    rng = np.random.default_rng(1)
    L = np.float32(1023.0)
    bins = rng.integers(0, 1023, size=(2000, 3))
    codes = oracle.morton((bins + 0.5).astype(np.float32), L)
    for b, c in zip(bins, codes):
        assert _decode_bits(c) == tuple(int(v) for v in b)


def test_morton_bins_follow_box_fraction():
    s = workloads.workload("lj_n4096_rho0.6")
    codes = oracle.morton(s.pos, s.L)
    got = np.array([_decode_bits(c) for c in codes])
    exact = np.floor(s.pos.astype(np.float64) * 1023.0 / float(s.L))
    assert got.max() <= 1022 and got.min() >= 0
    assert np.abs(got - np.minimum(exact, 1022)).max() <= 1
    # away from a bin edge the bin is forced
    frac = s.pos.astype(np.float64) * 1023.0 / float(s.L) - exact
    far = (frac > 1e-3) & (frac < 1 - 1e-3)
    assert (got[far] == exact[far]).all()


def _seg_setup(seed=0, n=3000, nseg=3):
    rng = np.random.default_rng(seed)
    L = np.float32(16.0)
    pos = rng.uniform(0, float(L), size=(n, 3)).astype(np.float32)
    seg = rng.integers(0, nseg, n).astype(np.int32)
    return pos, seg, np.full(nseg, L, np.float32)


def test_sort_is_stable_lexicographic():
    pos, seg, Ls = _seg_setup()
    # duplicate some positions so equal codes occur
    pos[100:200] = pos[100]
    t = oracle.lbvh_build(pos, seg, Ls)
    codes = oracle.morton(pos, Ls[0], seg, Ls)
    expect = np.lexsort((np.arange(pos.shape[0]), codes, seg))
    assert np.array_equal(t["order"], expect)
    assert np.array_equal(t["codes"], codes)


def _aug_key(codes_sorted, k):
    return (int(codes_sorted[k]) << 32) | k


def _prefix(a, b):
    x = a ^ b
    return 64 - x.bit_length()


def _check_tree(pos, seg, Ls):
    t = oracle.lbvh_topology(pos, seg, Ls)
    codes = oracle.morton(pos, Ls[0], seg, Ls)
    cs = codes[t["order"]]
    ss = t["seg_start"]
    for s in range(len(Ls)):
        a, b = int(ss[s]), int(ss[s + 1]) - 1
        if b <= a:
            if b == a:
                assert t["rope_leaf"][a] == END
            continue
        seen_int, parents = set(), {}
        stack = [a]
        while stack:
            k = stack.pop()
            assert k not in seen_int
            seen_int.add(k)
            f, l = int(t["first"][k]), int(t["last"][k])
            assert a <= f < l <= b
            # radix-tree property: the range is exactly the keys sharing the node's prefix
            d = _prefix(_aug_key(cs, f), _aug_key(cs, l))
            if f > a:
                assert _prefix(_aug_key(cs, f - 1), _aug_key(cs, f)) < d
            if l < b:
                assert _prefix(_aug_key(cs, l), _aug_key(cs, l + 1)) < d
            for c, side in ((int(t["left"][k]), 0), (int(t["right"][k]), 1)):
                if c >= 0:
                    cf, cl = int(t["first"][c]), int(t["last"][c])
                    assert c == (cl if side == 0 else cf)      # Karras numbering
                    stack.append(c)
                else:
                    cf = cl = ~c
                parents[(c, side)] = k
                # the left child holds the prefix followed by 0, the right by 1
                bit = 63 - d
                for m in (cf, cl):
                    assert (_aug_key(cs, m) >> bit) & 1 == side
            lf = t["first"][t["left"][k]] if t["left"][k] >= 0 else ~t["left"][k]
            rl_ = t["last"][t["right"][k]] if t["right"][k] >= 0 else ~t["right"][k]
            assert lf == f and rl_ == l
        assert len(seen_int) == b - a          # N - 1 internal nodes
    return t


def test_hierarchy_is_the_radix_tree_of_sorted_keys():
    pos, seg, Ls = _seg_setup(2, 2500, 4)
    _check_tree(pos, seg, Ls)


def test_hierarchy_with_many_equal_codes():
    pos, seg, Ls = _seg_setup(3, 1200, 1)
    pos[::3] = pos[5]
    pos[1::7] = np.float32(0.0)
    _check_tree(pos, seg, Ls)


def test_hierarchy_tiny_sizes():
    for n in (1, 2, 3, 4, 5, 17):
        pos, seg, Ls = _seg_setup(n, n, 1)
        _check_tree(pos, seg, Ls)


def _rope_walk(t, a, b, overlap):
    """Stackless traversal: descend on overlap, else follow the rope (Alg. 1)."""
    visits = []
    node = a if b > a else ~a
    while node != END:
        visits.append(node)
        if node >= 0 and overlap(node):
            node = int(t["left"][node])
        elif node >= 0:
            node = int(t["rope_int"][node])
        else:
            node = int(t["rope_leaf"][~node])
        assert len(visits) <= 2 * (b - a + 1)
    return visits


def _stack_dfs(t, a, b, overlap):
    visits = []
    stack = [a if b > a else ~a]
    while stack:
        node = stack.pop()
        visits.append(node)
        if node >= 0 and overlap(node):
            stack.append(int(t["right"][node]))
            stack.append(int(t["left"][node]))
    return visits


@pytest.mark.parametrize("p", [1.0, 0.0, 0.5, 0.9])
def test_rope_walk_equals_stack_based_dfs(p):
    pos, seg, Ls = _seg_setup(5, 1500, 2)
    t = oracle.lbvh_topology(pos, seg, Ls)
    rng = np.random.default_rng(11)
    mask = rng.random(pos.shape[0]) < p
    for s in range(2):
        a, b = int(t["seg_start"][s]), int(t["seg_start"][s + 1]) - 1
        ropes = _rope_walk(t, a, b, lambda k: mask[k])
        dfs = _stack_dfs(t, a, b, lambda k: mask[k])
        assert ropes == dfs
        if p == 1.0:
            assert len(ropes) == 2 * (b - a + 1) - 1       # every node once
        if p == 0.0:
            assert ropes == [a]


def _decoded(node_word_lo, node_word_hi, frame):
    qlo = oracle.unpack10(node_word_lo)
    qhi = oracle.unpack10(node_word_hi)
    lo, hi = oracle.dequantize(qlo, qhi, frame[:3], frame[3:])
    return lo, hi, qlo, qhi


def test_quantized_nodes_contain_their_particles_and_are_tight():
    s = workloads.workload("lj_n4096_rho0.6")
    seg = np.zeros(s.n, np.int32)
    t = oracle.lbvh_build(s.pos, seg, [s.L])
    topo = oracle.lbvh_topology(s.pos, seg, [s.L])
    fr = t["frame"][0]
    h = fr[3:].astype(np.float64)
    P = s.pos[t["order"]]
    assert np.array_equal(t["root"][0, :3], P.min(0)) and np.array_equal(t["root"][0, 3:], P.max(0))
    for k in range(s.n - 1):
        f, l = topo["first"][k], topo["last"][k]
        lo, hi, qlo, qhi = _decoded(t["nodes"][k, 0], t["nodes"][k, 1], fr)
        sub = P[f : l + 1]
        assert (lo <= sub.min(0)).all() and (hi >= sub.max(0)).all()
        # at most one bin (plus rounding) of slack on each face
        assert (sub.min(0) - lo <= h * 1.0001 + 1e-6).all()
        assert (hi - sub.max(0) <= h * 1.0001 + 1e-6).all()
        assert (qlo <= qhi).all() and (qhi <= 1023).all()
    lo, hi, qlo, qhi = _decoded(t["nodes"][0, 0], t["nodes"][0, 1], fr)
    assert qlo.tolist() == [0, 0, 0] and qhi.tolist() == [1023, 1023, 1023]


def _containment_failures(quantize, rng, trials=4000):
    bad = 0
    for _ in range(trials):
        R_lo = rng.uniform(-50, 50, 3).astype(np.float32)
        ext = (10.0 ** rng.uniform(-3, 3, 3)).astype(np.float32)
        R_hi = (R_lo + ext).astype(np.float32)
        h = np.zeros(3, np.float32)
        for d in range(3):   # frame as the oracle forms it: round-up (R_hi - R_lo) / 1023
            _, hh = _frame_of(R_lo[d], R_hi[d])
            h[d] = hh
        a = rng.uniform(R_lo, R_hi).astype(np.float32)
        b = rng.uniform(R_lo, R_hi).astype(np.float32)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        if rng.random() < 0.2:
            lo = R_lo.copy()
        if rng.random() < 0.2:
            hi = R_hi.copy()
        qlo, qhi = quantize(lo, hi, R_lo, h)
        dlo, dhi = oracle.dequantize(qlo, qhi, R_lo, h)
        if not ((dlo <= lo).all() and (dhi >= hi).all()):
            bad += 1
    return bad


def _frame_of(r_lo, r_hi):
    # same frame the oracle builds, obtained through a one-particle-pair tree
    pos = np.array([[r_lo, 0, 0], [r_hi, 0, 0]], np.float32)
    pos[:, 1:] = 0
    t = oracle.lbvh_build(pos, np.zeros(2, np.int32), [np.float32(1e6)])
    return t["frame"][0, 0], t["frame"][0, 3]


def test_outward_quantization_never_loses_volume():
    rng = np.random.default_rng(12)
    assert _containment_failures(oracle.quantize_box, rng) == 0


def test_containment_check_detects_round_to_nearest():
    # planted mistake: quantize with round-to-nearest instead of directed rounding
    def nearest(lo, hi, R_lo, h):
        ql = np.clip(np.rint((lo - R_lo) / h), 0, 1023).astype(np.uint32)
        qh = np.clip(np.rint((hi - R_lo) / h), 0, 1023).astype(np.uint32)
        return ql, qh
    rng = np.random.default_rng(12)
    assert _containment_failures(nearest, rng, trials=500) > 0


def test_degenerate_frame():
    pos = np.full((5, 3), 3.25, np.float32)
    t = oracle.lbvh_build(pos, np.zeros(5, np.int32), [np.float32(10)])
    fr = t["frame"][0]
    assert (fr[3:] == np.finfo(np.float32).tiny).all()
    for k in range(4):
        lo, hi, qlo, qhi = _decoded(t["nodes"][k, 0], t["nodes"][k, 1], fr)
        assert (qlo == 0).all() and (qhi == 0).all()
        assert (lo == 3.25).all() and (hi == 3.25).all()


@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_node_and_leaf_words(K):
    pos, seg, Ls = _seg_setup(9, 700, 2)
    t = oracle.lbvh_build(pos, seg, Ls, bundle_k=K)
    topo = oracle.lbvh_topology(pos, seg, Ls)
    assert np.array_equal(t["order"], topo["order"])
    for s in range(2):
        a, b = int(t["seg_start"][s]), int(t["seg_start"][s + 1]) - 1
        for k in range(a, b):
            w = t["nodes"][k]
            cnt = topo["last"][k] - topo["first"][k] + 1
            bundle = (int(w[0]) >> 31) & 1
            assert bundle == int(K >= 2 and cnt <= K)
            assert w[2] == (topo["first"][k] if bundle else topo["left"][k])
            assert w[3] == topo["rope_int"][k]
        for k in range(a, b + 1):
            lw = t["leaves"][k]
            assert np.array_equal(lw[:3], pos[t["order"][k]])
            tag = int(lw[3:4].view(np.uint32)[0])
            assert tag & 0x7FFFFFFF == t["order"][k]
            r = int(topo["rope_leaf"][k])
            assert (tag >> 31) == int(r >= 0)
            # a leaf's rope is always the node starting at the next leaf, or the end
            assert r == END if k == b else (r == k + 1 or r == ~(k + 1))


def _exact_width(r_lo, r_hi, bins):
    """Bin width (r_hi - r_lo) / bins in exact arithmetic, rounded up to FP32."""
    from fractions import Fraction
    x = (Fraction(float(r_hi)) - Fraction(float(r_lo))) / bins
    f = np.float32(float(x))
    if Fraction(float(f)) < x:
        f = np.nextafter(f, np.float32(np.inf))
    return f


def test_frame_width_21_bit_is_the_rounded_up_quotient():
    # 2^21 - 1 bins per axis: the width is the exact quotient rounded up (the
    # oracle forms the difference and the quotient under round-up in FP32)
    rng = np.random.default_rng(21)
    for _ in range(500):
        R_lo = rng.uniform(0, 100, 3).astype(np.float32)
        R_hi = (R_lo + (10.0 ** rng.uniform(-2, 2.5, 3))).astype(np.float32)
        h = oracle.frame_width(R_lo, R_hi, 21)
        for d in range(3):
            exact = _exact_width(R_lo[d], R_hi[d], 2 ** 21 - 1)
            # FP32 round-up of the difference first: never below the exact
            # quotient, at most two ulps above it
            assert h[d] >= exact and h[d] <= np.nextafter(np.nextafter(exact, np.float32(np.inf)),
                                                          np.float32(np.inf))
    assert (oracle.frame_width(np.zeros(3), np.zeros(3), 21) == np.finfo(np.float32).tiny).all()


def test_outward_quantization_21_bit_never_loses_volume_and_is_tight():
    rng = np.random.default_rng(22)
    bad = loose = 0
    for _ in range(3000):
        R_lo = rng.uniform(-50, 50, 3).astype(np.float32)
        R_hi = (R_lo + (10.0 ** rng.uniform(-2, 3, 3))).astype(np.float32)
        h = oracle.frame_width(R_lo, R_hi, 21)
        a = rng.uniform(R_lo, R_hi).astype(np.float32)
        b = rng.uniform(R_lo, R_hi).astype(np.float32)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        if rng.random() < 0.2:
            lo = R_lo.copy()
        if rng.random() < 0.2:
            hi = R_hi.copy()
        qlo, qhi = oracle.quantize_box(lo, hi, R_lo, h, bits=21)
        assert (qhi <= 2 ** 21 - 1).all() and (qlo <= qhi).all()
        dlo, dhi = oracle.dequantize(qlo, qhi, R_lo, h)
        bad += not ((dlo <= lo).all() and (dhi >= hi).all())
        # within two bins (plus FP32 rounding of the decode) of the box
        slack = 2 * h.astype(np.float64) + 4 * np.spacing(np.abs(R_hi).astype(np.float32)).astype(np.float64)
        loose += not ((lo - dlo <= slack).all() and (dhi - hi <= slack).all())
    assert bad == 0 and loose == 0


def test_21_bit_boxes_detect_a_frame_built_for_10_bits():
    # planted mistake: 21-bit codes decoded with the 10-bit bin width land far
    # outside the box they came from
    R_lo = np.zeros(3, np.float32)
    R_hi = np.full(3, 50.0, np.float32)
    h21 = oracle.frame_width(R_lo, R_hi, 21)
    h10 = oracle.frame_width(R_lo, R_hi, 10)
    lo = np.full(3, 20.0, np.float32)
    qlo, qhi = oracle.quantize_box(lo, lo, R_lo, h21, bits=21)
    dlo, dhi = oracle.dequantize(qlo, qhi, R_lo, h10)
    assert not ((dlo <= lo).all() and (dhi >= lo).all())
    dlo, dhi = oracle.dequantize(qlo, qhi, R_lo, h21)
    assert (dlo <= lo).all() and (dhi >= lo).all()
