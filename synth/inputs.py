"""Seeded synthetic inputs shaped like the paper's benchmark workloads.

This module is shared by the oracle side and the GPU side of every test and
benchmark.  It holds no finite-element arithmetic: it never computes node
positions, quadrature points, shape functions, row blocks or patterns.  It
only defines, as functions of *physical* points handed to it by the caller,

* the localisation centres of the orbitals (uniform or clustered blobs),
* the potential V(x) = -sum_j d * exp(-|x - a_j|^2 / (2 sigma^2)),
* the orbital field  phi_alpha(x) = g(key, alpha) * exp(-|x - c_alpha|^2 / s^2)
  restricted to the ball |x - c_alpha| <= R,

where g is a standard normal drawn from a counter-based generator keyed by
(seed, lattice key of the node, orbital id), so that every caller gets the
same number for the same node and orbital whatever order or subset it asks
for.  The generator is SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a
counter hash, followed by the Box-Muller transform.

The paper's workload is a (10,0) carbon nanotube with two orbitals per atom
and an 8 Bohr support radius (Sec. 4); the atom positions are not available,
so seeded centres in the box stand in for them, with the mesh sizes, orbital
counts, column-block counts and block fill of Tables 1 and 3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1907_01005


@dataclass(frozen=True)
class Config:
    """One synthetic workload.  Sizes are cells per direction and cell edge
    lengths; `p` is the polynomial degree of the Q_p elements."""

    name: str
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    p: int
    n_orb: int
    n_col_blocks: int
    radius: float          # support radius R of every orbital
    env_s2: float          # s^2 of the Gaussian envelope exp(-|x-c|^2/s^2)
    n_wells: int
    well_depth: float
    well_sigma: float
    centres: str = "uniform"          # "uniform" or "blobs"
    n_blobs: int = 8
    dirichlet: int = 1
    index: int = 0                    # config index used in the seed
    target_fill: float | None = None  # intended block fill of the pattern
    notes: str = ""

    @property
    def box(self):
        return (self.nx * self.hx, self.ny * self.hy, self.nz * self.hz)

    @property
    def seed(self) -> int:
        return SEED_BASE + 1000 * self.index


def _cfg(**kw) -> Config:
    return Config(**kw)


# R values below were chosen so that the closed (one-cell dilated) block
# pattern reaches the target fill; tests/test_oracle_pins.py checks the
# fill with the oracle's own pattern builder.
CONFIGS: dict[str, Config] = {
    # Tiny FP64 case: unit cube, 4x4x4 Q2 cells (729 DoFs), 16 orbitals in two
    # column blocks of 8, R = 0.35, envelope exp(-|x-c|^2/0.04), four wells of
    # depth 1 and width 0.15.
    "tiny": _cfg(name="tiny", nx=4, ny=4, nz=4, hx=0.25, hy=0.25, hz=0.25, p=2,
                 n_orb=16, n_col_blocks=2, radius=0.35, env_s2=0.04,
                 n_wells=4, well_depth=1.0, well_sigma=0.15, index=0),
    # Same tiny box with Q4 cells (two per direction), for p=4 parity at small size.
    "tiny_p4": _cfg(name="tiny_p4", nx=2, ny=2, nz=2, hx=0.5, hy=0.5, hz=0.5, p=4,
                    n_orb=16, n_col_blocks=2, radius=0.35, env_s2=0.04,
                    n_wells=4, well_depth=1.0, well_sigma=0.15, index=5),
    # Small cases that span many tiles, with partly empty patterns and ragged
    # column blocks (widths 1..16), used for element-by-element parity.
    "small_p2": _cfg(name="small_p2", nx=12, ny=8, nz=10, hx=1.0, hy=0.75, hz=1.25, p=2,
                     n_orb=61, n_col_blocks=7, radius=2.2, env_s2=(2.2 / 1.75) ** 2,
                     n_wells=6, well_depth=1.0, well_sigma=1.5, index=6),
    "small_p4": _cfg(name="small_p4", nx=8, ny=6, nz=6, hx=2.0, hy=1.5, hz=2.5, p=4,
                     n_orb=45, n_col_blocks=5, radius=2.5, env_s2=(2.5 / 1.75) ** 2,
                     n_wells=6, well_depth=1.0, well_sigma=1.5, index=7),
    "small_p1": _cfg(name="small_p1", nx=14, ny=10, nz=8, hx=0.5, hy=0.5, hz=0.5, p=1,
                     n_orb=33, n_col_blocks=4, radius=0.8, env_s2=(0.8 / 1.75) ** 2,
                     n_wells=3, well_depth=1.0, well_sigma=0.6, index=8),
    "small_p3": _cfg(name="small_p3", nx=8, ny=8, nz=6, hx=1.0, hy=1.0, hz=1.0, p=3,
                     n_orb=40, n_col_blocks=5, radius=1.2, env_s2=(1.2 / 1.75) ** 2,
                     n_wells=3, well_depth=1.0, well_sigma=1.0, index=9),
    "wide_p2": _cfg(name="wide_p2", nx=8, ny=8, nz=6, hx=1.0, hy=1.0, hz=1.0, p=2,
                    n_orb=48, n_col_blocks=3, radius=2.0, env_s2=(2.0 / 1.75) ** 2,
                    n_wells=4, well_depth=1.0, well_sigma=1.0, index=10),
    "narrow_p2": _cfg(name="narrow_p2", nx=8, ny=6, nz=6, hx=1.0, hy=1.0, hz=1.0, p=2,
                      n_orb=7, n_col_blocks=3, radius=1.8, env_s2=(1.8 / 1.75) ** 2,
                      n_wells=4, well_depth=1.0, well_sigma=1.0, index=11),
    "narrow_p4": _cfg(name="narrow_p4", nx=4, ny=4, nz=6, hx=2.0, hy=2.0, hz=2.0, p=4,
                      n_orb=5, n_col_blocks=5, radius=3.0, env_s2=(3.0 / 1.75) ** 2,
                      n_wells=4, well_depth=1.0, well_sigma=1.0, index=12),
    # Natural (free) boundary: boundary nodes carry DoFs like interior ones.
    "free_p2": _cfg(name="free_p2", nx=8, ny=6, nz=4, hx=1.0, hy=1.0, hz=1.0, p=2,
                    n_orb=29, n_col_blocks=4, radius=1.8, env_s2=(1.8 / 1.75) ** 2,
                    n_wells=4, well_depth=1.0, well_sigma=1.0, dirichlet=0, index=13),
    "free_p4": _cfg(name="free_p4", nx=4, ny=4, nz=2, hx=2.0, hy=2.0, hz=2.0, p=4,
                    n_orb=21, n_col_blocks=3, radius=3.0, env_s2=(3.0 / 1.75) ** 2,
                    n_wells=4, well_depth=1.0, well_sigma=1.0, dirichlet=0, index=14),
    # Wide unions at small size: supports large against the box, so that runs
    # of consecutive row blocks hold well over 128 columns between them
    # (several 128-column output tiles of the Gram per group, mirrored
    # off-diagonal tiles, row splits), at sizes the oracle checks in full.
    "multi_p2": _cfg(name="multi_p2", nx=12, ny=8, nz=8, hx=1.0, hy=1.0, hz=1.0, p=2,
                     n_orb=200, n_col_blocks=24, radius=3.4, env_s2=(3.4 / 1.75) ** 2,
                     n_wells=6, well_depth=1.0, well_sigma=1.5, index=15),
    "multi_p4": _cfg(name="multi_p4", nx=6, ny=4, nz=4, hx=2.0, hy=2.0, hz=2.0, p=4,
                     n_orb=200, n_col_blocks=24, radius=3.4, env_s2=(3.4 / 1.75) ** 2,
                     n_wells=6, well_depth=1.0, well_sigma=1.5, index=16),
    # 16-wide column blocks whose unions exceed 256 columns.
    "multi_w16_p2": _cfg(name="multi_w16_p2", nx=10, ny=8, nz=6, hx=1.0, hy=1.0, hz=1.0, p=2,
                         n_orb=320, n_col_blocks=20, radius=4.0, env_s2=(4.0 / 1.75) ** 2,
                         n_wells=4, well_depth=1.0, well_sigma=1.5, index=17),
    # Paper scale, p=2: 64x40x40 unit Q2 cells = 102,400 cells, 846,369 DoFs,
    # 12,800 row blocks; 320 orbitals in 38 column blocks; ~20% block fill;
    # 50 wells of depth 1 and width 2 cells.
    "p2": _cfg(name="p2", nx=64, ny=40, nz=40, hx=1.0, hy=1.0, hz=1.0, p=2,
               n_orb=320, n_col_blocks=38, radius=11.35, env_s2=(11.35 / 1.75) ** 2,
               n_wells=50, well_depth=1.0, well_sigma=2.0, index=1, target_fill=0.20),
    # Paper scale, p=4: the same domain one level coarser (32x20x20 Q4 cells of
    # edge 2), 12,800 cells, 846,369 DoFs, 1,600 row blocks, ~15% block fill.
    "p4": _cfg(name="p4", nx=32, ny=20, nz=20, hx=2.0, hy=2.0, hz=2.0, p=4,
               n_orb=320, n_col_blocks=38, radius=7.6, env_s2=(7.6 / 1.75) ** 2,
               n_wells=50, well_depth=1.0, well_sigma=2.0, index=2, target_fill=0.15),
    # Larger: 1,686,177 DoFs, 640 orbitals drawn from 8 Gaussian blobs, 70 blocks.
    "large_p2": _cfg(name="large_p2", nx=128, ny=40, nz=40, hx=1.0, hy=1.0, hz=1.0, p=2,
                     n_orb=640, n_col_blocks=70, radius=7.5, env_s2=(7.5 / 1.75) ** 2,
                     n_wells=100, well_depth=1.0, well_sigma=2.0, centres="blobs",
                     index=3),
    "large_p4": _cfg(name="large_p4", nx=64, ny=20, nz=20, hx=2.0, hy=2.0, hz=2.0, p=4,
                     n_orb=640, n_col_blocks=70, radius=7.5, env_s2=(7.5 / 1.75) ** 2,
                     n_wells=100, well_depth=1.0, well_sigma=2.0, centres="blobs",
                     index=4),
}


def get_config(name: str) -> Config:
    return CONFIGS[name]


def scaled_config(base: Config, name: str, **changes) -> Config:
    """A copy of `base` with some fields replaced (used by the serving mix)."""
    d = {k: getattr(base, k) for k in base.__dataclass_fields__}
    d.update(changes)
    d["name"] = name
    return Config(**d)


# ---------------------------------------------------------------------------
# Counter-based normal generator: SplitMix64 as a hash, then Box-Muller.
# ---------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_ORB = np.uint64(0xD1B54A32D192ED03)


def _splitmix64_mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (finaliser) on uint64 arrays."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def counter_normals(seed: int, key: np.ndarray, orbital: np.ndarray) -> np.ndarray:
    """Standard normal N(0,1) for each (key, orbital) pair, a pure function of
    (seed, key, orbital).  `key` is a non-negative integer node key (the lattice
    index), `orbital` the original orbital id."""
    key = np.asarray(key, dtype=np.uint64)
    orbital = np.asarray(orbital, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = (np.uint64(seed) * _GOLDEN) ^ (key * _GOLDEN) ^ ((orbital + np.uint64(1)) * _ORB)
        z1 = _splitmix64_mix(base + _GOLDEN)
        z2 = _splitmix64_mix(base + _GOLDEN + _GOLDEN)
    # 53-bit uniforms in (0, 1]
    u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------------------
# Orbital centres and potential wells
# ---------------------------------------------------------------------------
def orbital_centres(cfg: Config) -> np.ndarray:
    """(n_orb, 3) centres: uniform in the box, or drawn from n_blobs Gaussian
    blobs of width box/8 (clipped into the box)."""
    rng = np.random.default_rng(cfg.seed + 11)
    L = np.array(cfg.box)
    if cfg.centres == "uniform":
        return rng.uniform(0.0, 1.0, size=(cfg.n_orb, 3)) * L
    blob_c = rng.uniform(0.15, 0.85, size=(cfg.n_blobs, 3)) * L
    which = rng.integers(0, cfg.n_blobs, size=cfg.n_orb)
    c = blob_c[which] + rng.normal(size=(cfg.n_orb, 3)) * (L / 8.0)
    return np.clip(c, 0.0, L * (1.0 - 1e-12))


def well_centres(cfg: Config) -> np.ndarray:
    rng = np.random.default_rng(cfg.seed + 23)
    return rng.uniform(0.0, 1.0, size=(cfg.n_wells, 3)) * np.array(cfg.box)


def potential(cfg: Config, xyz: np.ndarray, chunk: int = 1 << 18) -> np.ndarray:
    """V(x) = -sum_j d exp(-|x - a_j|^2 / (2 sigma^2)) at points xyz (n,3), FP64."""
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    a = well_centres(cfg)
    out = np.empty(len(xyz))
    inv = 1.0 / (2.0 * cfg.well_sigma ** 2)
    for s in range(0, len(xyz), chunk):
        x = xyz[s:s + chunk]
        d2 = ((x[:, None, :] - a[None, :, :]) ** 2).sum(-1)
        out[s:s + chunk] = -cfg.well_depth * np.exp(-d2 * inv).sum(-1)
    return out


def orbital_support(cfg: Config, xyz: np.ndarray, alpha: int,
                    centres: np.ndarray | None = None) -> np.ndarray:
    """Boolean mask of the points xyz (n,3) inside the support ball of orbital
    `alpha`: |x - c_alpha| <= R."""
    c = (orbital_centres(cfg) if centres is None else centres)[alpha]
    d2 = ((np.asarray(xyz, dtype=np.float64) - c) ** 2).sum(-1)
    return d2 <= cfg.radius ** 2


def orbital_values(cfg: Config, xyz: np.ndarray, key: np.ndarray, alpha: int,
                   centres: np.ndarray | None = None) -> np.ndarray:
    """phi_alpha at points xyz (n,3) with node keys `key` (n,):
    N(0,1)(seed, key, alpha) * exp(-|x - c|^2 / s^2); zero outside the ball."""
    c = (orbital_centres(cfg) if centres is None else centres)[alpha]
    xyz = np.asarray(xyz, dtype=np.float64)
    d2 = ((xyz - c) ** 2).sum(-1)
    g = counter_normals(cfg.seed, key, np.full(len(xyz), alpha))
    v = g * np.exp(-d2 / cfg.env_s2)
    v[d2 > cfg.radius ** 2] = 0.0
    return v


def support_candidates(cfg: Config, alpha: int, centres: np.ndarray | None = None):
    """Axis-aligned bounding box [lo, hi] of the support ball of `alpha`, so
    callers can restrict the points they evaluate."""
    c = (orbital_centres(cfg) if centres is None else centres)[alpha]
    return c - cfg.radius, c + cfg.radius


# ---------------------------------------------------------------------------
# Serving request mix
# ---------------------------------------------------------------------------
SERVING_MESHES = ((16, 10, 10), (32, 20, 20), (64, 40, 40))


def serving_config(index: int, mesh: tuple, p: int, n_orb: int, fill: float) -> Config:
    """One serving request workload: a box of `mesh` cells of edge 1 for p = 2;
    for p = 4 half as many cells per direction (rounded up to even) of edge
    2, so both degrees cover about the same domain with the same DoF count),
    `n_orb` uniform orbitals in column blocks of
    about 8.4, and a support radius sized from the target block fill by a
    ball-volume estimate (the actual fill is what the pattern builder finds).
    """
    h = 1.0 if p <= 2 else 2.0
    nx, ny, nz = mesh
    if p > 2:                                   # half the cells per direction, rounded up to even
        nx, ny, nz = (2 * max(1, (n + 3) // 4) for n in (nx, ny, nz))
    vol = nx * ny * nz * h ** 3
    patch = 2.0 * h
    r = (fill * vol * 3.0 / (4.0 * math.pi)) ** (1.0 / 3.0) - 2.0 * patch
    r = max(r, 1.5 * h)
    ncb = max(1, int(round(n_orb / 8.42)))
    return Config(name=f"serve{index}", nx=nx, ny=ny, nz=nz, hx=h, hy=h, hz=h, p=p, n_orb=n_orb,
                  n_col_blocks=ncb, radius=r, env_s2=(r / 1.75) ** 2, n_wells=max(4, nx * ny * nz // 2000),
                  well_depth=1.0, well_sigma=2.0 * h, index=100 + index, target_fill=fill)


def serving_mix(n: int, seed: int = SEED_BASE + 7, meshes=SERVING_MESHES, degrees=(2, 4),
                orb_range=(32, 640), fill_range=(0.10, 0.30)):
    """n request workloads drawn from the serving mix: the meshes taken in
    turn (so that a small pool holds every mesh size), degree uniform over
    the given set, orbital count log-uniform, fill uniform."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        mesh = meshes[i % len(meshes)]
        p = int(degrees[int(rng.integers(len(degrees)))])
        m = int(round(math.exp(rng.uniform(math.log(orb_range[0]), math.log(orb_range[1])))))
        f = float(rng.uniform(*fill_range))
        out.append(serving_config(i, mesh, p, m, f))
    return out


def poisson_arrivals(n: int, rate_per_s: float, seed: int = SEED_BASE + 9) -> np.ndarray:
    """Arrival offsets (s) of a Poisson stream of n requests."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
