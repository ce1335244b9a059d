"""Pins for the FP64 Lennard-Jones oracle (Eq. 1, truncated and shifted at r_c).

Checked against hand-worked values (golden), the simple-cubic lattice sum over
coordination shells, Newton's third law, linearity of U in eps, invariance
under a joint scaling of lengths, and FP64 central finite differences for the
forces and both parameter gradients.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _pair(r, L=20.0):
    pos = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]], np.float64)
    return pos


def _eval_pair(r, eps=1.0, sig=1.0, rc=2.5):
    p64 = _pair(r)
    p32 = p64.astype(np.float32)
    rows = np.array([[1], [0]], np.int32)
    counts = np.array([1, 1], np.int32)
    return oracle.lj_fp64(p32, np.zeros(2, np.int32), np.float32(20.0), [[eps]], [[sig]],
                          np.float32(rc), rows, counts, pos64=p64)


def test_golden_pair_values():
    gold = json.load(open(os.path.join(GOLD, "lj_values.json")))
    for c in gold["cases"]:
        r = c["r"] if "r" in c else eval(c["r_expr"], {}, {})
        out = _eval_pair(r)
        # U counts the pair once (1/2 from each row)
        assert out["U"] == pytest.approx(c["u"], abs=1e-12)
        assert out["F"][0, 0] == pytest.approx(c["F0x"], abs=1e-9)
        assert out["F"][1, 0] == pytest.approx(-c["F0x"], abs=1e-9)
        assert out["e"][0] == pytest.approx(0.5 * c["u"], abs=1e-12)


def test_shift_vanishes_at_cutoff():
    out = _eval_pair(np.nextafter(np.float32(2.5), np.float32(0)).astype(np.float64))
    assert abs(out["U"]) < 1e-8
    out = _eval_pair(2.6)   # beyond r_c: no interaction
    assert out["U"] == 0.0 and not out["F"].any()


def _sc_lattice(m, a):
    g = (np.arange(m, dtype=np.float64) + 0.5) * a
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.float32), np.float32(m * a)


def test_simple_cubic_lattice_sum():
    pos, L = _sc_lattice(6, 1.0)
    rc = 2.5
    rows, counts = oracle.nlist(pos, L, rc, method="brute", cap=128)
    out = oracle.lj_fp64(pos, np.zeros(len(pos), np.int32), L, [[1.0]], [[1.0]],
                         np.float32(rc), rows, counts)

    def u(r):
        return 4 * (r ** -12 - r ** -6) - 4 * (rc ** -12 - rc ** -6)
    shells = [(6, 1.0), (12, 2 ** 0.5), (8, 3 ** 0.5), (6, 2.0), (24, 5 ** 0.5), (24, 6 ** 0.5)]
    per_particle = 0.5 * sum(z * u(r) for z, r in shells)
    assert out["U"] / len(pos) == pytest.approx(per_particle, rel=1e-12)
    assert np.abs(out["F"]).max() < 1e-12            # perfect lattice: no net force


def _two_type_system(n=1500, seed=4):
    s = workloads.jittered_lattice(n, 0.8, 0.3, seed, r_cut=2.5, skin=0.3)
    rng = np.random.default_rng(seed)
    types = (rng.random(s.n) < 0.5).astype(np.int32)
    rows, counts = oracle.nlist(s.pos, s.L, s.r_list[0, 0], method="cell")
    E = np.array([[1.0, 1.5], [1.5, 0.5]])
    S = np.array([[1.0, 0.88], [0.88, 0.8]])
    return s, types, rows, counts, E, S


def test_newton_third_law_and_eps_linearity():
    s, types, rows, counts, E, S = _two_type_system()
    out = oracle.lj_fp64(s.pos, types, s.L, E, S, np.float32(2.5), rows, counts)
    scale = np.abs(out["F"]).sum()
    assert np.abs(out["F"].sum(0)).max() < 1e-11 * scale
    # U is linear in every eps entry: sum eps * dU/deps = U
    assert (E * out["dE"]).sum() == pytest.approx(out["U"], rel=1e-12)


def test_joint_length_scaling_leaves_energy_unchanged():
    s, types, rows, counts, E, S = _two_type_system(800, 5)
    base = oracle.lj_fp64(s.pos, types, s.L, E, S, np.float32(2.5), rows, counts)
    lam = 2.0   # exact in binary: positions, L, sigma and r_c scale without rounding
    out = oracle.lj_fp64(s.pos * np.float32(lam), types, s.L * np.float32(lam), E, S * lam,
                         np.float32(2.5 * lam), rows, counts)
    assert out["U"] == pytest.approx(base["U"], rel=1e-12)


def test_finite_differences_forces_and_parameter_gradients():
    s, types, rows, counts, E, S = _two_type_system(1000, 6)
    rc = np.float32(2.5)
    p64 = s.pos.astype(np.float64)
    base = oracle.lj_fp64(s.pos, types, s.L, E, S, rc, rows, counts, pos64=p64)
    rng = np.random.default_rng(0)

    def central(i, a, h):
        pp, pm = p64.copy(), p64.copy()
        pp[i, a] += h
        pm[i, a] -= h
        up = oracle.lj_fp64(s.pos, types, s.L, E, S, rc, rows, counts, pos64=pp)["U"]
        um = oracle.lj_fp64(s.pos, types, s.L, E, S, rc, rows, counts, pos64=pm)["U"]
        return (up - um) / (2 * h)

    h = 1e-4
    for _ in range(64):
        i, a = int(rng.integers(s.n)), int(rng.integers(3))
        # Richardson extrapolation of the central differences at h and h/2 cancels
        # the h^2 truncation term, which is large for the close pairs of a
        # jittered lattice
        fd = -(4 * central(i, a, h / 2) - central(i, a, h)) / 3
        f = base["F"][i, a]
        assert abs(fd - f) <= 1e-6 * max(1.0, abs(f)), (i, a, fd, f)
    for name, P in (("dE", E), ("dS", S)):
        for a in range(2):
            for b in range(2):
                hp = 1e-6
                Pp, Pm = P.copy(), P.copy()
                Pp[a, b] += hp
                Pm[a, b] -= hp
                kw = dict(pos64=p64)
                if name == "dE":
                    up = oracle.lj_fp64(s.pos, types, s.L, Pp, S, rc, rows, counts, **kw)["U"]
                    um = oracle.lj_fp64(s.pos, types, s.L, Pm, S, rc, rows, counts, **kw)["U"]
                else:
                    up = oracle.lj_fp64(s.pos, types, s.L, E, Pp, rc, rows, counts, **kw)["U"]
                    um = oracle.lj_fp64(s.pos, types, s.L, E, Pm, rc, rows, counts, **kw)["U"]
                fd = (up - um) / (2 * hp)
                g = base[name][a, b]
                assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (name, a, b, fd, g)
