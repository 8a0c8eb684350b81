"""Seeded synthetic inputs and MeshBlock layouts.

This module holds no arithmetic of the compact-FD method: it only draws
random parameters, evaluates smooth analytic test fields (and their exact
derivatives, for error reports) at cell-centred sample points, and builds
block lists with their 26-neighbour tables.  Both the CUDA path and the
oracle consume what it produces.

Field layout used everywhere: a float array of shape
(nblocks, nfields, E, E, E) per block size, E = N + 2 g, axes (z, y, x), x
fastest.  Blocks of different sizes are concatenated in block order.

Cell-centred sampling (Eq. gridDisc, CC): local interior index k of a block
with origin index o (in units of its dx) sits at x = (o + k + 1/2) dx; ghost
indices k in [-g, 0) and [N, N + g) continue the same formula.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Dict, List, Sequence, Tuple

import numpy as np

TWO_PI = 2.0 * np.pi

# Neighbour directions (dz, dy, dx) in {-1,0,1}^3 without the centre,
# lexicographic order (dz slowest).  Index r in [0, 26).
DIRS: Tuple[Tuple[int, int, int], ...] = tuple(
    (dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dz, dy, dx) != (0, 0, 0))


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# Analytic fields
# ---------------------------------------------------------------------------


@dataclass
class SineSum:
    """f = sum_j A_j sin(k_j . x + phi_j) with integer wavevectors (periodic on [0, 2pi)^3)."""

    k: np.ndarray      # (n, 3) as (kx, ky, kz)
    A: np.ndarray
    phi: np.ndarray

    def __call__(self, x, y, z):
        out = 0.0
        for (kx, ky, kz), A, p in zip(self.k, self.A, self.phi):
            out = out + A * np.sin(kx * x + ky * y + kz * z + p)
        return out

    def deriv(self, op: str, x, y, z):
        """Exact derivative for op in dx, dy, dz, dxx, ..., dyz."""
        idx = {"x": 0, "y": 1, "z": 2}
        out = 0.0
        for kv, A, p in zip(self.k, self.A, self.phi):
            arg = kv[0] * x + kv[1] * y + kv[2] * z + p
            fac = 1.0
            for c in op[1:]:
                fac = fac * kv[idx[c]]
            n = len(op) - 1
            base = (np.cos(arg), -np.sin(arg))[n - 1] if n == 1 else -np.sin(arg)
            out = out + A * fac * base
        return out


def sine_sum(r: np.random.Generator, n: int = 8, kmin: int = 1, kmax: int = 12) -> SineSum:
    """Seeded sine sum: integer k in [kmin, kmax]^3, A ~ U(-1, 1), phi ~ U[0, 2pi)."""
    k = r.integers(kmin, kmax + 1, size=(n, 3))
    A = r.uniform(-1.0, 1.0, size=n)
    phi = r.uniform(0.0, TWO_PI, size=n)
    return SineSum(k, A, phi)


def sine_sum_ball(r: np.random.Generator, n: int, kmax_norm: float) -> SineSum:
    """Integer wavevectors drawn uniformly from {k : 1 <= |k| <= kmax_norm}, random signs."""
    K = int(np.floor(kmax_norm))
    g = np.arange(-K, K + 1)
    cand = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    nrm = np.sqrt((cand ** 2).sum(1))
    cand = cand[(nrm >= 1) & (nrm <= kmax_norm)]
    k = cand[r.integers(0, len(cand), size=n)]
    A = r.uniform(-1.0, 1.0, size=n)
    phi = r.uniform(0.0, TWO_PI, size=n)
    return SineSum(k, A, phi)


@dataclass
class PeriodicGaussian:
    """exp(-|x - c|^2 / (2 sigma^2)) summed over the 27 periodic images (shifts 0, +-2pi)."""

    c: np.ndarray
    sigma: float

    def __call__(self, x, y, z):
        out = 0.0
        for sz in (-1, 0, 1):
            for sy in (-1, 0, 1):
                for sx in (-1, 0, 1):
                    r2 = ((x - self.c[0] - sx * TWO_PI) ** 2 + (y - self.c[1] - sy * TWO_PI) ** 2
                          + (z - self.c[2] - sz * TWO_PI) ** 2)
                    out = out + np.exp(-r2 / (2.0 * self.sigma ** 2))
        return out


def gaussian(r: np.random.Generator, width: float = 0.1) -> PeriodicGaussian:
    """Gaussian bump of width ``width`` x domain (sigma = width * 2pi), seeded centre."""
    return PeriodicGaussian(r.uniform(0.0, TWO_PI, size=3), width * TWO_PI)


@dataclass
class InverseDistance:
    """sum_p 1/(|x - x_p| + 0.5), |.| the periodic minimum-image distance."""

    centers: np.ndarray  # (n, 3)

    def __call__(self, x, y, z):
        out = 0.0
        for c in self.centers:
            d2 = 0.0
            for v, cc in zip((x, y, z), c):
                dv = np.abs(v - cc) % TWO_PI
                dv = np.minimum(dv, TWO_PI - dv)
                d2 = d2 + dv * dv
            out = out + 1.0 / (np.sqrt(d2) + 0.5)
        return out


@dataclass
class Sum:
    parts: List[Callable]

    def __call__(self, x, y, z):
        out = 0.0
        for p in self.parts:
            out = out + p(x, y, z)
        return out


# ---------------------------------------------------------------------------
# MeshBlock layouts
# ---------------------------------------------------------------------------


@dataclass
class Mesh:
    """Block list: size N_b, origin index (ox, oy, oz) in units of dx_b, spacing, neighbours."""

    n: np.ndarray          # (nb,) interior points per axis
    origin: np.ndarray     # (nb, 3) as (ox, oy, oz)
    dx: np.ndarray         # (nb, 3) as (dx, dy, dz)
    neighbors: np.ndarray  # (nb, 26) int32, -1 = caller fills that ghost region
    g: int
    shape: Tuple[int, ...] = field(default=())  # (nbz, nby, nbx) for uniform meshes

    @property
    def nblocks(self) -> int:
        return len(self.n)

    def ext(self, b: int) -> int:
        return int(self.n[b]) + 2 * self.g

    def coords(self, b: int):
        """Ghost-extended sample coordinates (x, y, z) 1D arrays of block b."""
        E = np.arange(-self.g, int(self.n[b]) + self.g) + 0.5
        return tuple((self.origin[b, a] + E) * self.dx[b, a] for a in range(3))


def uniform_mesh(NM: int, N: int, g: int = 4, L: float = TWO_PI) -> Mesh:
    """Periodic NM^3 grid on [0, L)^3 as (NM/N)^3 blocks of N^3, block index (bz*nb + by)*nb + bx."""
    nb = NM // N
    assert nb * N == NM and g <= N
    idx = np.arange(nb ** 3)
    bz, by, bx = idx // (nb * nb), (idx // nb) % nb, idx % nb
    origin = np.stack([bx * N, by * N, bz * N], 1)
    neighbors = np.empty((nb ** 3, 26), np.int32)
    for r, (dz, dy, dxx) in enumerate(DIRS):
        neighbors[:, r] = (((bz + dz) % nb) * nb + (by + dy) % nb) * nb + (bx + dxx) % nb
    dx = np.full((nb ** 3, 3), L / NM)
    return Mesh(np.full(nb ** 3, N), origin, dx, neighbors, g, (nb, nb, nb))


def periodic_box_mesh(nbx: int, nby: int, nbz: int, N: int, g: int = 4, L: float = TWO_PI) -> Mesh:
    """Periodic box of nbx x nby x nbz blocks of N^3 with spacing L / (nbx N) on every axis (a
    2D problem is a box one block thick in z); block index (bz*nby + by)*nbx + bx."""
    idx = np.arange(nbx * nby * nbz)
    bz, by, bx = idx // (nbx * nby), (idx // nbx) % nby, idx % nbx
    origin = np.stack([bx * N, by * N, bz * N], 1)
    neighbors = np.empty((len(idx), 26), np.int32)
    for r, (dz, dy, dxx) in enumerate(DIRS):
        neighbors[:, r] = (((bz + dz) % nbz) * nby + (by + dy) % nby) * nbx + (bx + dxx) % nbx
    dx = np.full((len(idx), 3), L / (nbx * N))
    return Mesh(np.full(len(idx), N), origin, dx, neighbors, g, (nbz, nby, nbx))


def box_in_box_mesh(g: int = 4) -> Mesh:
    """448 blocks of 16^3 and 64 of 32^3 on [0, 2pi)^3.

    Seven octants of side pi at coarse spacing pi/64 (4^3 blocks of 16^3
    each) and the octant [0, pi)^3 refined 2:1 (spacing pi/128, 4^3 blocks of
    32^3).  Coarse blocks come first.  Faces, edges and corners between blocks
    of the same size are periodic neighbours; a region that touches the other
    level gets -1 (its ghosts are filled by sampling the analytic field).
    """
    nc = 8                      # coarse blocks per axis over the whole domain
    ns, ds = [], []
    origins = []
    coarse_index = {}
    fine_index = {}
    for bz in range(nc):
        for by in range(nc):
            for bx in range(nc):
                if bx < 4 and by < 4 and bz < 4:
                    continue    # inside the refined octant
                coarse_index[(bz, by, bx)] = len(ns)
                ns.append(16)
                origins.append((bx * 16, by * 16, bz * 16))
                ds.append(np.pi / 64)
    for bz in range(4):
        for by in range(4):
            for bx in range(4):
                fine_index[(bz, by, bx)] = len(ns)
                ns.append(32)
                origins.append((bx * 32, by * 32, bz * 32))
                ds.append(np.pi / 128)
    nbk = len(ns)
    nbr = np.full((nbk, 26), -1, np.int32)
    for (bz, by, bx), b in coarse_index.items():
        for r, (dz, dy, dxx) in enumerate(DIRS):
            key = ((bz + dz) % nc, (by + dy) % nc, (bx + dxx) % nc)
            nbr[b, r] = coarse_index.get(key, -1)
    for (bz, by, bx), b in fine_index.items():
        for r, (dz, dy, dxx) in enumerate(DIRS):
            key = (bz + dz, by + dy, bx + dxx)
            nbr[b, r] = fine_index.get(key, -1)   # outside the octant: other level
    dx = np.repeat(np.asarray(ds)[:, None], 3, 1)
    return Mesh(np.asarray(ns), np.asarray(origins), dx, nbr, g)


def sample(mesh: Mesh, fields: Sequence[Callable], dtype=np.float64, blocks=None) -> List[np.ndarray]:
    """Evaluate fields on every block's ghost-extended points.

    Returns one array per distinct consecutive run of block sizes is not
    needed by callers; instead a list with one (nfields, E, E, E) array per
    block is returned (ghosts filled analytically everywhere).
    """
    out = []
    bl = range(mesh.nblocks) if blocks is None else blocks
    for b in bl:
        x, y, z = mesh.coords(b)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        out.append(np.stack([np.asarray(f(X, Y, Z), dtype=np.float64) for f in fields]).astype(dtype))
    return out


def pack(blocks: List[np.ndarray]) -> np.ndarray:
    """Concatenate per-block (nfields, E, E, E) arrays into one flat buffer."""
    return np.concatenate([b.reshape(-1) for b in blocks])


def unpack(flat: np.ndarray, mesh: Mesh, nfields: int, interior: bool = False, nops: int = 0):
    """Inverse of ``pack`` (interior=False) or split a (nops) interior output buffer."""
    out, off = [], 0
    for b in range(mesh.nblocks):
        n = int(mesh.n[b])
        if interior:
            cnt = nfields * nops * n ** 3
            out.append(flat[off:off + cnt].reshape(nfields, nops, n, n, n))
        else:
            E = n + 2 * mesh.g
            cnt = nfields * E ** 3
            out.append(flat[off:off + cnt].reshape(nfields, E, E, E))
        off += cnt
    return out


# ---------------------------------------------------------------------------
# The five benchmark workloads
# ---------------------------------------------------------------------------


def workload_fields(config: int, seed: int | None = None):
    """Analytic fields of each workload (seed = 2302 + config by default)."""
    r = rng(2302 + config if seed is None else seed)
    if config == 1:
        return [sine_sum(r, 8, 1, 12)]
    if config in (2, 3):
        return [sine_sum(r, 8, 1, 12), sine_sum(r, 8, 1, 12), gaussian(r, 0.1), gaussian(r, 0.1)]
    if config == 4:
        out = []
        for _ in range(22):
            inv = InverseDistance(r.uniform(0.0, TWO_PI, size=(2, 3)))
            out.append(Sum([sine_sum_ball(r, 8, 16.0), inv]))
        return out
    raise ValueError(config)


@dataclass
class PlaneWaves:
    """Phi = sum_j A_j cos(k_j . x - w_j t + phi_j), w_j = |k_j|: exact u_tt = Laplacian u."""

    k: np.ndarray
    A: np.ndarray
    phi: np.ndarray

    def phi_at(self, t, x, y, z):
        out = 0.0
        for kv, A, p in zip(self.k, self.A, self.phi):
            w = np.sqrt((kv ** 2).sum())
            out = out + A * np.cos(kv[0] * x + kv[1] * y + kv[2] * z - w * t + p)
        return out

    def K_at(self, t, x, y, z):
        out = 0.0
        for kv, A, p in zip(self.k, self.A, self.phi):
            w = np.sqrt((kv ** 2).sum())
            out = out + A * w * np.sin(kv[0] * x + kv[1] * y + kv[2] * z - w * t + p)
        return out


def plane_waves(seed: int = 2307, n: int = 8, kmax_norm: float = 20.0) -> PlaneWaves:
    s = sine_sum_ball(rng(seed), n, kmax_norm)
    return PlaneWaves(s.k, s.A, s.phi)
