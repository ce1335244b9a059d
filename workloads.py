"""Seeded synthetic particle configurations for the neighbor-search workloads.

This module only *creates inputs*: positions, types, box edges and cutoffs.
It holds none of the neighbor-search arithmetic, so both the CPU oracle and
the CUDA path can use it without sharing any of the method.

The paper measures on molecular-dynamics snapshots of Lennard-Jones and WCA
fluids in cubic periodic boxes with rho = N / L^3 (Sec. 4); those snapshots are
not published, so seeded stand-ins with the same shapes are generated here:

* ``jittered_lattice``  -- simple-cubic lattice with uniform per-axis jitter
  (LJ fluid stand-in, Sec. 4.1).
* ``binary_mixture``    -- large spheres by random sequential addition plus a
  uniform small-particle solvent outside their cores (size-asymmetric
  mixture, the case the paper's introduction motivates BVHs with, Sec. 1).
* ``batched_ensemble``  -- many independent jittered-lattice systems of
  uneven N and density.
* ``two_type_lj``       -- jittered lattice with a 50/50 random type split.
* ``jittered_lattice64`` -- the jittered lattice kept in double precision
  (the paper's double-precision particle data, Sec. 2.2, Sec. 4.1-4.2).
* ``spinodal_like``     -- an inhomogeneous liquid/vapor configuration, the
  stand-in for the paper's spinodal-decomposition snapshots (Sec. 4.3).

Conventions (all generators):
* FP64 arithmetic, rounded to float32 once at the end.
* The box edge is ``L = float32((N / rho) ** (1/3))``; the float32 value is
  authoritative for everything downstream.
* Positions lie in ``[0, L)``: coordinates are wrapped in FP64 with the float32
  L, rounded, and a coordinate that rounds up to L is mapped to 0 (its
  periodic image).
* Randomness comes from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "System",
    "System64",
    "jittered_lattice64",
    "pack_double4",
    "WCA_RCUT",
    "spinodal_like",
    "box_edge",
    "jittered_lattice",
    "binary_mixture",
    "batched_ensemble",
    "two_type_lj",
    "pack_float4",
    "workload",
    "WORKLOADS",
]


@dataclass
class System:
    """One periodic particle configuration.

    pos   : float32 [N, 3], every coordinate in [0, L)
    types : int32 [N], values in [0, n_types)
    L     : float32 cubic box edge
    r_list: float32 [n_types, n_types] symmetric list radius (r_cut + skin)
    r_cut : float32 [n_types, n_types] potential cutoff (<= r_list)
    """

    pos: np.ndarray
    types: np.ndarray
    L: np.float32
    n_types: int
    r_list: np.ndarray
    r_cut: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


@dataclass
class System64:
    """One periodic configuration with double-precision particle data.

    pos   : float64 [N, 3], every coordinate in [0, L)
    types : int32 [N], values in [0, n_types)
    L     : float (FP64) cubic box edge, authoritative
    r_list: float32 [n_types, n_types] list radius (r_cut + skin)
    r_cut : float32 [n_types, n_types]
    """

    pos: np.ndarray
    types: np.ndarray
    L: float
    n_types: int
    r_list: np.ndarray
    r_cut: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


# WCA cutoff: LJ truncated at its minimum, r_c = 2^(1/6) sigma (Sec. 4.2)
WCA_RCUT = float(2.0 ** (1.0 / 6.0))


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def box_edge(n: int, rho: float) -> np.float32:
    """Cubic box edge for n particles at number density rho, rounded once to FP32."""
    return np.float32((n / rho) ** (1.0 / 3.0))


def _wrap_to_f32(x64: np.ndarray, L: np.float32) -> np.ndarray:
    """Wrap FP64 coordinates into [0, L) with the FP32 box edge, round to FP32."""
    Ld = float(L)
    w = np.mod(x64, Ld)
    out = w.astype(np.float32)
    out[out >= L] = np.float32(0.0)
    out[out < 0] = np.float32(0.0)
    return out


def _matrix(n_types: int, value) -> np.ndarray:
    m = np.asarray(value, dtype=np.float32)
    if m.ndim == 0:
        m = np.full((n_types, n_types), m, dtype=np.float32)
    return np.ascontiguousarray(m.astype(np.float32))


def _lattice_f64(n: int, L: float, jitter: float, rng):
    """FP64 jittered simple-cubic sites (unwrapped) and the sites per axis."""
    m = int(round(n ** (1.0 / 3.0)))
    if m ** 3 < n:
        m += 1
    while (m - 1) ** 3 >= n and m > 1:
        m -= 1
    a = float(L) / m
    if m ** 3 == n:
        sites = np.arange(n, dtype=np.int64)
    else:
        sites = np.sort(rng.permutation(m ** 3)[:n])
    ix = sites // (m * m)
    iy = (sites // m) % m
    iz = sites % m
    base = (np.stack([ix, iy, iz], axis=1).astype(np.float64) + 0.5) * a
    jit = rng.uniform(-jitter, jitter, size=(n, 3))
    return base + jit, m, a


def jittered_lattice(n: int, rho: float, jitter: float, seed,
                     r_cut: float = 3.0, skin: float = 0.3) -> System:
    """Simple-cubic lattice with per-axis uniform jitter in [-jitter, +jitter].

    m = ceil(N^(1/3)) sites per axis with spacing a = L / m; when m^3 > N a
    seeded permutation picks which N sites are occupied.
    """
    if n <= 0:
        raise ValueError("n must be positive")
    rng = _rng(seed)
    L = box_edge(n, rho)
    x64, m, a = _lattice_f64(n, float(L), jitter, rng)
    pos = _wrap_to_f32(x64, L)
    rl = np.float32(r_cut) + np.float32(skin)
    return System(pos=np.ascontiguousarray(pos), types=np.zeros(n, np.int32), L=L,
                  n_types=1, r_list=_matrix(1, rl), r_cut=_matrix(1, r_cut),
                  meta=dict(kind="jittered_lattice", n=n, rho=rho, jitter=jitter,
                            seed=seed, sites_per_axis=m, spacing=a))


def jittered_lattice64(n: int, rho: float, jitter: float, seed,
                       r_cut: float = 3.0, skin: float = 0.3) -> System64:
    """The jittered lattice in double precision: L = (N / rho)^(1/3) in FP64
    (not rounded to FP32), positions wrapped into [0, L) in FP64.  The list
    radius is the FP32 value of r_cut + skin."""
    if n <= 0:
        raise ValueError("n must be positive")
    rng = _rng(seed)
    L = float((n / rho) ** (1.0 / 3.0))
    x64, m, a = _lattice_f64(n, L, jitter, rng)
    pos = np.mod(x64, L)
    pos[pos >= L] = 0.0
    pos[pos < 0] = 0.0
    rl = np.float32(np.float32(r_cut) + np.float32(skin))
    return System64(pos=np.ascontiguousarray(pos), types=np.zeros(n, np.int32), L=L,
                    n_types=1, r_list=_matrix(1, rl), r_cut=_matrix(1, r_cut),
                    meta=dict(kind="jittered_lattice64", n=n, rho=rho, jitter=jitter,
                              seed=seed, sites_per_axis=m, spacing=a))


def spinodal_like(n: int = 1_000_000, rho: float = 0.2, seed=0, rho_liquid: float = 0.72,
                  rho_vapor: float = 0.02, wavelength: float = 20.0, n_waves: int = 64,
                  r_cut: float = 3.0, skin: float = 0.0, double: bool = False):
    """Liquid/vapor stand-in for an LJ fluid quenched into the spinodal region
    (Sec. 4.3: N = 10^6 at rho = 0.2, quenched to T = 0.8, where it splits into
    liquid and vapor).  The domain pattern is Cahn's random-wave model of
    spinodal structures: the sign of a sum of n_waves plane waves of one
    wavelength with random directions and phases.  The field is thresholded so
    that liquid fills the volume fraction the lever rule gives,
    (rho - rho_vapor) / (rho_liquid - rho_vapor).  Liquid regions take the
    sites of a jittered lattice at rho_liquid (jitter half the spacing); the
    remaining particles are uniform in the vapor region, so N is exact.
    Returns a System (FP32) or, with double=True, a System64.
    """
    rng = _rng(seed)
    L64 = (n / rho) ** (1.0 / 3.0)
    L32 = np.float32(L64)
    L = float(L32) if not double else L64
    kdir = rng.normal(size=(n_waves, 3))
    kvec = kdir / np.linalg.norm(kdir, axis=1, keepdims=True) * (2.0 * np.pi / wavelength)
    # periodic box: snap the wave vectors onto the box's reciprocal lattice
    kvec = np.round(kvec * L / (2.0 * np.pi)) * (2.0 * np.pi / L)
    phase = rng.uniform(0.0, 2.0 * np.pi, n_waves)

    def field(x):
        out = np.zeros(x.shape[0])
        for k in range(0, n_waves, 8):
            out += np.cos(x @ kvec[k:k + 8].T + phase[k:k + 8]).sum(1)
        return out

    phi = (rho - rho_vapor) / (rho_liquid - rho_vapor)
    probe = rng.uniform(0.0, L, size=(200_000, 3))
    thr = np.quantile(field(probe), 1.0 - phi)
    # liquid: jittered lattice at rho_liquid over the box, sites in the liquid region
    m = int(np.ceil((rho_liquid * L ** 3) ** (1.0 / 3.0)))
    a = L / m
    g = (np.arange(m, dtype=np.float64) + 0.5) * a
    sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    sites = sites + rng.uniform(-0.5 * a, 0.5 * a, size=sites.shape)
    liquid = sites[field(sites) > thr]
    if liquid.shape[0] > n:
        liquid = liquid[np.sort(rng.permutation(liquid.shape[0])[:n])]
    # vapor: uniform in the rest of the box up to exactly n particles
    vap = []
    need = n - liquid.shape[0]
    while need > 0:
        cand = rng.uniform(0.0, L, size=(max(4 * need, 1024), 3))
        cand = cand[field(cand) <= thr][:need]
        vap.append(cand)
        need -= cand.shape[0]
    x = np.concatenate([liquid] + vap, 0)
    x = x[rng.permutation(n)]
    if double:
        pos = np.mod(x, L)
        pos[pos >= L] = 0.0
        pos[pos < 0] = 0.0
        rl = np.float32(np.float32(r_cut) + np.float32(skin))
        return System64(pos=np.ascontiguousarray(pos), types=np.zeros(n, np.int32), L=L, n_types=1,
                        r_list=_matrix(1, rl), r_cut=_matrix(1, r_cut),
                        meta=dict(kind="spinodal_like", n=n, rho=rho, n_liquid=int(liquid.shape[0])))
    pos = _wrap_to_f32(x, L32)
    rl = np.float32(r_cut) + np.float32(skin)
    return System(pos=np.ascontiguousarray(pos), types=np.zeros(n, np.int32), L=L32, n_types=1,
                  r_list=_matrix(1, rl), r_cut=_matrix(1, r_cut),
                  meta=dict(kind="spinodal_like", n=n, rho=rho, n_liquid=int(liquid.shape[0])))


def _periodic_d2(a: np.ndarray, b: np.ndarray, L: float) -> np.ndarray:
    """FP64 squared minimum-image distance between rows of a [k,3] and b [3]."""
    d = a - b
    d -= L * np.rint(d / L)
    return np.einsum("ij,ij->i", d, d)


def binary_mixture(seed, L: float = 100.0, n_large: int = 400, d_large: float = 10.0,
                   rho_small: float = 0.5, core_radius: float = 5.0,
                   n_small: int | None = None, skin: float = 0.4,
                   r_cut_ss: float = 3.0, r_cut_sl: float = 5.5,
                   r_cut_ll: float = 10.0) -> System:
    """Size-asymmetric binary mixture in a cubic periodic box.

    Large spheres (type 1) are placed by random sequential addition with
    centre separation >= d_large (periodic).  Small particles (type 0) are
    uniform in the free volume outside radius ``core_radius`` of every large
    centre.  With the defaults the free volume is 1e6 - 400 * 4/3 pi 5^3 and
    the small count is round(rho_small * free volume) = 395,280.
    """
    rng = _rng(seed)
    Lf = np.float32(L)
    Ld = float(Lf)
    centres = np.empty((0, 3), np.float64)
    attempts = 0
    while centres.shape[0] < n_large:
        attempts += 1
        if attempts > 10_000_000:
            raise RuntimeError("random sequential addition did not converge")
        c = rng.uniform(0.0, Ld, size=3)
        if centres.shape[0] == 0 or _periodic_d2(centres, c, Ld).min() >= d_large ** 2:
            centres = np.vstack([centres, c])
    if n_small is None:
        free = Ld ** 3 - n_large * (4.0 / 3.0) * math.pi * core_radius ** 3
        n_small = int(round(rho_small * free))
    # rejection sampling against the large cores with a coarse cell grid
    nc = max(1, int(Ld // (2 * core_radius)))
    cw = Ld / nc
    cell_of = np.floor(centres / cw).astype(np.int64) % nc
    buckets: dict = {}
    for k, c in enumerate(cell_of):
        buckets.setdefault(tuple(c), []).append(k)
    out = []
    have = 0
    while have < n_small:
        cand = rng.uniform(0.0, Ld, size=(max(2 * (n_small - have), 4096), 3))
        ok = np.ones(cand.shape[0], bool)
        ccell = np.floor(cand / cw).astype(np.int64) % nc
        for off in np.ndindex(3, 3, 3):
            nb = (ccell + np.array(off) - 1) % nc
            keys = nb[:, 0] * nc * nc + nb[:, 1] * nc + nb[:, 2]
            for key in np.unique(keys):
                kk = (int(key // (nc * nc)), int((key // nc) % nc), int(key % nc))
                if kk not in buckets:
                    continue
                sel = np.nonzero(keys == key)[0]
                for k in buckets[kk]:
                    d2 = _periodic_d2(cand[sel], centres[k], Ld)
                    ok[sel[d2 < core_radius ** 2]] = False
        acc = cand[ok][: n_small - have]
        out.append(acc)
        have += acc.shape[0]
    small = np.vstack(out)
    pos64 = np.vstack([small, centres])
    pos = _wrap_to_f32(pos64, Lf)
    types = np.concatenate([np.zeros(n_small, np.int32), np.ones(n_large, np.int32)])
    rc = np.array([[r_cut_ss, r_cut_sl], [r_cut_sl, r_cut_ll]], np.float32)
    rl = (rc + np.float32(skin)).astype(np.float32)
    return System(pos=np.ascontiguousarray(pos), types=types, L=Lf, n_types=2,
                  r_list=rl, r_cut=rc,
                  meta=dict(kind="binary_mixture", seed=seed, n_small=n_small,
                            n_large=n_large, d_large=d_large, core_radius=core_radius))


def batched_ensemble(seed, n_sys: int = 256, n_min: int = 500, n_max: int = 50_000,
                     rho_min: float = 0.3, rho_max: float = 0.9, jitter: float = 0.3,
                     r_cut: float = 2.5, skin: float = 0.3) -> list[System]:
    """Independent jittered-lattice systems, N log-uniform, rho uniform.

    System k draws its own generator from (seed, k) so that any single system
    can be regenerated without the others.
    """
    rng = _rng(seed)
    logn = rng.uniform(math.log(n_min), math.log(n_max), size=n_sys)
    ns = np.clip(np.rint(np.exp(logn)).astype(np.int64), n_min, n_max)
    rhos = rng.uniform(rho_min, rho_max, size=n_sys)
    systems = []
    for k in range(n_sys):
        s = jittered_lattice(int(ns[k]), float(rhos[k]), jitter, seed=(seed, k),
                             r_cut=r_cut, skin=skin)
        s.meta["system"] = k
        systems.append(s)
    return systems


def two_type_lj(seed, n_sys: int = 32, n: int = 65_536, rho: float = 0.8,
                jitter: float = 0.3, r_cut: float = 2.5, skin: float = 0.3,
                eps=(1.0, 1.5, 0.5), sig=(1.0, 0.88, 0.8)) -> list[System]:
    """Two-type (50/50) jittered-lattice systems with per-pair LJ parameters.

    eps and sig are given in (AA, AB, BB) order and expanded to symmetric
    2x2 matrices stored in ``meta``.
    """
    systems = []
    E = np.array([[eps[0], eps[1]], [eps[1], eps[2]]], np.float64)
    S = np.array([[sig[0], sig[1]], [sig[1], sig[2]]], np.float64)
    for k in range(n_sys):
        s = jittered_lattice(n, rho, jitter, seed=(seed, k), r_cut=r_cut, skin=skin)
        rng = _rng((seed, k, 1))
        types = np.zeros(n, np.int32)
        types[rng.permutation(n)[: n // 2]] = 1
        s.types = types
        s.n_types = 2
        s.r_list = _matrix(2, np.float32(r_cut) + np.float32(skin))
        s.r_cut = _matrix(2, r_cut)
        s.meta.update(kind="two_type_lj", system=k, eps=E, sig=S)
        systems.append(s)
    return systems


def pack_float4(pos: np.ndarray, types: np.ndarray) -> np.ndarray:
    """[N,3] float32 + [N] int32 -> [N,4] float32 with w holding the type's int bits."""
    n = pos.shape[0]
    out = np.zeros((n, 4), np.float32)
    out[:, :3] = pos
    out.view(np.int32)[:, 3] = types.astype(np.int32)
    return out


def pack_double4(pos: np.ndarray, types: np.ndarray) -> np.ndarray:
    """[N,3] float64 + [N] int32 -> [N,4] float64 with w holding the type as a whole number."""
    n = pos.shape[0]
    out = np.zeros((n, 4), np.float64)
    out[:, :3] = pos
    out[:, 3] = types.astype(np.float64)
    return out


# Named workloads: the five configurations the build is measured and checked on.
def _lj4096(seed=0):
    return jittered_lattice(4096, 0.6, 0.3, seed, r_cut=3.0, skin=0.4)


def _lj2m(seed=0):
    return jittered_lattice(2_097_152, 0.8, 0.25, seed, r_cut=3.0, skin=0.3)


WORKLOADS = {
    "lj_n4096_rho0.6": _lj4096,
    "lj_n2097152_rho0.8": _lj2m,
    "mixture_L100": lambda seed=0: binary_mixture(seed),
    "ensemble_256": lambda seed=0: batched_ensemble(seed),
    "lj2type_32x65536": lambda seed=0: two_type_lj(seed),
    "spinodal_n1000000": lambda seed=0: spinodal_like(1_000_000, 0.2, seed),
}


def workload(name: str, seed=0):
    return WORKLOADS[name](seed)
