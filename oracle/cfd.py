"""FP64 block operators of arXiv 2302.14858, written for checking, not speed.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Conventions
-----------
* A centred compact scheme of derivative degree d is given by ``Sch``:
  ``a`` = alpha^{(d)}_{-1} = alpha^{(d)}_{+1} (alpha^{(d)}_0 = 1), ``rhs`` =
  alpha^{(0)}_{-M..M} and ``closure`` = alpha-bar^{(0)}_{-h..h} of the
  explicit closure C-bar_{p+1} (h = p + 1).
* A block holds N interior samples per axis and g ghost layers.  Local
  index k = 0..N-1 are the interior nodes (k*_- = 0, k*_+ = N-1); a pencil
  of ghost-extended data is stored with array index j = k + g, j = 0..N+2g-1.
* Cell-centred sampling (Eq. gridDisc, CC): x_k = a_I + (k + 1/2) dx.
* Sums over stencil offsets run left to right, m = -M .. M, in FP64 with
  separate multiply and add (no fused operations), then the sum is scaled by
  dx^{-d}.
* Pencils are the trailing axes of every array: the routines are vectorised
  over independent pencils only; each pencil's arithmetic is the textbook
  sequence written below.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, Iterable, List, Sequence, Tuple

import numpy as np

OPS = ("dx", "dy", "dz", "dxx", "dyy", "dzz", "dxy", "dxz", "dyz")
# axis letter -> array axis of a (z, y, x) block
_AX = {"z": 0, "y": 1, "x": 2}


@dataclass(frozen=True)
class Sch:
    """Centred tridiagonal compact scheme with its explicit closure."""

    d: int
    a: float
    rhs: Tuple[float, ...]
    closure: Tuple[float, ...]

    @property
    def M(self) -> int:
        return (len(self.rhs) - 1) // 2

    @property
    def h(self) -> int:
        return (len(self.closure) - 1) // 2


# ---------------------------------------------------------------------------
# 1D building blocks
# ---------------------------------------------------------------------------


def stencil_sum(f: np.ndarray, coeffs: Sequence[float], k0: int, k1: int, g: int) -> np.ndarray:
    """sum_{m=-H}^{H} c_m f_{k+m} for k = k0..k1-1 (local indices).

    ``f`` has the ghost-extended index j = k + g on axis 0.  Left-to-right
    order over m, separate multiply and add.
    """
    H = (len(coeffs) - 1) // 2
    acc = None
    for i, c in enumerate(coeffs):
        m = i - H
        term = c * f[k0 + m + g:k1 + m + g]
        acc = term if acc is None else acc + term
    return acc


def thomas(lo: np.ndarray, di: np.ndarray, up: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Thomas algorithm (tridiagonal LU without pivoting).

    Row k reads lo[k] x[k-1] + di[k] x[k] + up[k] x[k+1] = r[k]; the
    coefficient vectors have length n and r has shape (n, ...).
    """
    n = r.shape[0]
    c = np.zeros(n)
    dp = np.empty_like(r)
    den = di[0]
    c[0] = up[0] / den
    dp[0] = r[0] / den
    for k in range(1, n):
        den = di[k] - lo[k] * c[k - 1]
        if k < n - 1:
            c[k] = up[k] / den
        dp[k] = (r[k] - lo[k] * dp[k - 1]) / den
    x = np.empty_like(r)
    x[n - 1] = dp[n - 1]
    for k in range(n - 2, -1, -1):
        x[k] = dp[k] - c[k] * x[k + 1]
    return x


def closed_solve(f: np.ndarray, s: Sch, dx: float, N: int, g: int) -> np.ndarray:
    """Per-block system of Eq. sch_cent_om.

    Rows k = k*_- (0) and k*_+ (N-1) are the explicit closure
    d_k = dx^{-d} sum_m alpha-bar_m f_{k+m}; rows k = 1..N-2 are the interior
    scheme a d_{k-1} + d_k + a d_{k+1} = dx^{-d} sum_m alpha_m f_{k+m}.  The
    whole N x N tridiagonal system (closure rows as unit rows) is solved by
    the Thomas algorithm.  ``f`` has shape (N + 2g, ...); returns (N, ...).
    """
    assert g >= s.h and g >= s.M
    scale = 1.0 / dx ** s.d
    r = np.empty((N,) + f.shape[1:])
    r[0] = stencil_sum(f, s.closure, 0, 1, g)[0] * scale
    r[N - 1] = stencil_sum(f, s.closure, N - 1, N, g)[0] * scale
    r[1:N - 1] = stencil_sum(f, s.rhs, 1, N - 1, g) * scale
    lo = np.full(N, s.a)
    up = np.full(N, s.a)
    di = np.ones(N)
    lo[0] = up[0] = 0.0
    lo[N - 1] = up[N - 1] = 0.0
    return thomas(lo, di, up, r)


def iterated_solve(f: np.ndarray, s: Sch, dx: float, N: int, g: int,
                   d_lo: np.ndarray, d_hi: np.ndarray) -> np.ndarray:
    """One hybrid iteration, Eq. iter_center_P (reading of the garbled row).

    Unknowns run over k = k^c_- .. k^c_+ with k^c_- = k*_- - 2 = -2 and
    k^c_+ = k*_+ + 2 = N + 1.  Rows k^c_+- fix the derivative to the previous
    iterate at that global point (``d_lo``, ``d_hi``: values communicated from
    the neighbouring blocks); rows k = -1 .. N are the interior scheme
    a d_{k-1} + d_k + a d_{k+1} = dx^{-d} sum_m alpha_m f_{k+m}.  Returns the N
    interior values k = 0..N-1.
    """
    assert g >= s.M + 1
    n = N + 4
    scale = 1.0 / dx ** s.d
    r = np.empty((n,) + f.shape[1:])
    r[0] = d_lo
    r[n - 1] = d_hi
    r[1:n - 1] = stencil_sum(f, s.rhs, -1, N + 1, g) * scale
    lo = np.full(n, s.a)
    up = np.full(n, s.a)
    di = np.ones(n)
    lo[0] = up[0] = 0.0
    lo[n - 1] = up[n - 1] = 0.0
    return thomas(lo, di, up, r)[2:N + 2]


def cyclic_matrices(s: Sch, n: int, dx: float) -> Tuple[np.ndarray, np.ndarray]:
    """Global periodic scheme as dense circulant matrices (A, B) with A d = B f."""
    A = np.zeros((n, n))
    B = np.zeros((n, n))
    for k in range(n):
        A[k, k] = 1.0
        A[k, (k - 1) % n] += s.a
        A[k, (k + 1) % n] += s.a
        for i, c in enumerate(s.rhs):
            B[k, (k + i - s.M) % n] += c / dx ** s.d
    return A, B


def global_periodic(f: np.ndarray, s: Sch, dx: float) -> np.ndarray:
    """Undecomposed periodic scheme along axis 0 (the "global scheme").

    The cyclic tridiagonal system is solved with a library dense solve.
    """
    n = f.shape[0]
    A, B = cyclic_matrices(s, n, dx)
    rhs = B @ f.reshape(n, -1)
    return np.linalg.solve(A, rhs).reshape(f.shape)


# ---------------------------------------------------------------------------
# Ghost fill: the communication matrix G of Eq. example_G
# ---------------------------------------------------------------------------


def ghost_fill_1d(fg: np.ndarray, N: int, g: int) -> np.ndarray:
    """Split a periodic global line into blocks with g ghosts on each side.

    Block I holds global indices I N - g .. I N + N + g - 1 (mod N_M): its
    interior is its own data and its ghosts come from I-1 and I+1 mod N_S.
    Returns shape (N_S, N + 2g, ...).
    """
    NM = fg.shape[0]
    NS = NM // N
    idx = (np.arange(NS)[:, None] * N + np.arange(-g, N + g)[None, :]) % NM
    return fg[idx]


def ghost_fill_3d(fg: np.ndarray, N: int, g: int) -> np.ndarray:
    """Uniform periodic 3D decomposition of a global (z, y, x) array.

    Returns (nbz, nby, nbx, E, E, E), E = N + 2g, ghosts (faces, edges and
    corners) filled from the periodic neighbours.
    """
    nz, ny, nx = fg.shape
    iz = ghost_fill_1d(np.arange(nz), N, g)
    iy = ghost_fill_1d(np.arange(ny), N, g)
    ix = ghost_fill_1d(np.arange(nx), N, g)
    return fg[iz[:, None, None, :, None, None], iy[None, :, None, None, :, None],
              ix[None, None, :, None, None, :]]


def exchange_ghosts(blocks: List[np.ndarray], neighbors: np.ndarray, N: int, g: int) -> List[np.ndarray]:
    """Fill every ghost region of every block by copying the neighbour's interior.

    ``blocks[b]`` is a (E, E, E) array (z, y, x).  ``neighbors[b, r]`` is the
    neighbour in direction r, r enumerating (dz, dy, dx) in {-1,0,1}^3 without
    (0,0,0) in lexicographic order; -1 leaves that region untouched.  Ghost
    cell (z, y, x) of region (dz, dy, dx) takes the neighbour's value at
    (z - dz N, y - dy N, x - dx N) (local interior coordinates).  Same-size
    neighbours only.
    """
    out = [b.copy() for b in blocks]
    dirs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
            if (dz, dy, dx) != (0, 0, 0)]

    def rng(dd):
        return {-1: range(-g, 0), 0: range(0, N), 1: range(N, N + g)}[dd]

    for b in range(len(blocks)):
        for r, (dz, dy, dx) in enumerate(dirs):
            nb = neighbors[b][r]
            if nb < 0:
                continue
            for z in rng(dz):
                for y in rng(dy):
                    for x in rng(dx):
                        out[b][z + g, y + g, x + g] = blocks[nb][z - dz * N + g, y - dy * N + g, x - dx * N + g]
    return out


# ---------------------------------------------------------------------------
# Decomposed 1D operator with hybrid iteration
# ---------------------------------------------------------------------------


def decomposed_1d(fg: np.ndarray, s: Sch, dx: float, N: int, g: int, n_iter: int) -> np.ndarray:
    """Derivative of a periodic line under domain decomposition.

    [0]: closed per-block solve (Eq. sch_cent_om).  [i], i >= 1: every block
    re-solves with Eq. iter_center_P using the [i-1] values of its neighbours
    at its k^c_+- nodes (Jacobi style: all blocks read iterate i-1).
    """
    ext = ghost_fill_1d(fg, N, g)               # (NS, E, ...)
    NS = ext.shape[0]
    d = np.stack([closed_solve(ext[I], s, dx, N, g) for I in range(NS)])
    for _ in range(n_iter):
        prev = d
        d = np.stack([
            iterated_solve(ext[I], s, dx, N, g, prev[(I - 1) % NS][N - 2], prev[(I + 1) % NS][1])
            for I in range(NS)])
    return d.reshape((NS * N,) + fg.shape[1:])


# ---------------------------------------------------------------------------
# Embedded dense operators (Sec. "Embedded operations")
# ---------------------------------------------------------------------------


def embedded_G(NS: int, N: int, g: int) -> np.ndarray:
    """Block-partitioned communication matrix G (Eq. example_G)."""
    E = N + 2 * g
    G = np.zeros((NS * E, NS * E))
    for I in range(NS):
        for j in range(E):
            k = j - g
            if 0 <= k < N:
                src_block, src = I, j
            elif k < 0:
                src_block, src = (I - 1) % NS, k + N + g
            else:
                src_block, src = (I + 1) % NS, k - N + g
            G[I * E + j, src_block * E + src] = 1.0
    return G


def embedded_D0(s: Sch, N: int, g: int, dx: float) -> np.ndarray:
    """[0]D = dx^{-d} (D-bar_L)^{-1} D-bar_R on one ghost-extended block.

    D-bar_L (Eq. diff_mat_subL): unit rows on ghosts and at k*_+-, tridiagonal
    rows in between.  D-bar_R (Eq. diff_mat_subR): closure stencil at k*_+-,
    interior stencil in between; its ghost rows are set to zero here (they
    are overwritten by the G applied afterwards).
    """
    E = N + 2 * g
    L = np.eye(E)
    R = np.zeros((E, E))
    for k in range(N):
        j = k + g
        if k in (0, N - 1):
            for i, c in enumerate(s.closure):
                R[j, j + i - s.h] = c
        else:
            L[j, j - 1] = s.a
            L[j, j + 1] = s.a
            for i, c in enumerate(s.rhs):
                R[j, j + i - s.M] = c
    return np.linalg.solve(L, R) / dx ** s.d


def embedded_iteration_parts(s: Sch, N: int, g: int):
    """D_L, D_R (Eq. diff_mat_subMR), E^c_+-, Z^c_- Z^c_+ on one block.

    Local (ghost-extended) indices: k^c_- = g - 2, k^c_+ = g + N + 1.
    """
    E = N + 2 * g
    kcm, kcp = g - 2, g + N + 1
    L = np.eye(E)
    R = np.eye(E)
    for j in range(kcm + 1, kcp):
        L[j, j - 1] = s.a
        L[j, j + 1] = s.a
        R[j, :] = 0.0
        for i, c in enumerate(s.rhs):
            R[j, j + i - s.M] = c
    Em = np.zeros((E, E)); Em[kcm, kcm] = 1.0
    Ep = np.zeros((E, E)); Ep[kcp, kcp] = 1.0
    Zm = np.zeros((E, E)); Zp = np.zeros((E, E))
    for j in range(kcm, kcp + 1):
        Zm[j, j] = 1.0
        Zp[j, j] = 1.0
    Zm[kcm, kcm] = 0.0
    Zp[kcp, kcp] = 0.0
    return L, R, Em, Ep, Zm @ Zp


def embedded_operator(s: Sch, NS: int, N: int, g: int, dx: float, i: int) -> np.ndarray:
    """[i]D of Eq. iter_scheme for a periodic line of NS blocks."""
    G = embedded_G(NS, N, g)
    D0 = embedded_D0(s, N, g, dx)
    Dk = G @ np.kron(np.eye(NS), D0) @ G
    if i == 0:
        return Dk
    L, R, Em, Ep, Z = embedded_iteration_parts(s, N, g)
    Linv = np.kron(np.eye(NS), np.linalg.inv(L))
    ZR = np.kron(np.eye(NS), Z @ R) / dx ** s.d
    EE = np.kron(np.eye(NS), Em + Ep)
    for _ in range(i):
        Dk = G @ (Linv @ (ZR + EE @ Dk))
    return Dk


# ---------------------------------------------------------------------------
# 3D application
# ---------------------------------------------------------------------------


def _axis_solve(data: np.ndarray, axis: int, s: Sch, dx: float, N: int, g: int,
                n_iter: int, block_axis: int | None) -> np.ndarray:
    """Solve along local ``axis`` (0, 1, 2 of the last three dims) of ``data``.

    ``data`` has shape (nbz, nby, nbx, e0, e1, e2) with extent N + 2g along
    ``axis``; the result has extent N there.  With n_iter > 0 the neighbour
    along ``block_axis`` (0, 1, 2 of the first three dims, periodic) supplies
    the k^c values.
    """
    ax = 3 + axis
    f = np.moveaxis(data, ax, 0)
    d = closed_solve(f, s, dx, N, g)
    for _ in range(n_iter):
        prev = d
        lo = np.roll(prev, 1, axis=1 + block_axis)[N - 2]
        hi = np.roll(prev, -1, axis=1 + block_axis)[1]
        d = iterated_solve(f, s, dx, N, g, lo, hi)
    return np.moveaxis(d, 0, ax)


def apply_uniform(ext: np.ndarray, s1: Sch, s2: Sch, dx3: Sequence[float], N: int, g: int,
                  ops: Iterable[str] = OPS, n_iter: int = 0) -> Dict[str, np.ndarray]:
    """All requested derivatives on a uniform periodic block decomposition.

    ``ext`` is (nbz, nby, nbx, E, E, E) with ghosts filled (Eq. example_G);
    ``dx3`` = (dx_x, dx_y, dx_z).  Single-axis ops use the d = 1 scheme ``s1``
    or the d = 2 scheme ``s2``.  Mixed ops follow Sec. "Z4c: system
    description": d_ij -> (D_i[D_j f] + D_j[D_i f]) / 2, each inner D_j
    evaluated locally on the rows of the i-ghost zone (those use the edge
    ghosts), then D_i applied to that intermediate.  Returns interior arrays
    (nbz, nby, nbx, N, N, N) per op.
    """
    dxs = {"x": dx3[0], "y": dx3[1], "z": dx3[2]}
    I = slice(g, g + N)
    out = {}

    def solve(data, letter, sch):
        a = _AX[letter]
        return _axis_solve(data, a, sch, dxs[letter], N, g, n_iter, a)

    def interior_except(data, keep):
        sl = [slice(None)] * 3 + [I, I, I]
        for letter in keep:
            sl[3 + _AX[letter]] = slice(None)
        return data[tuple(sl)]

    for op in ops:
        if len(op) == 2:
            c = op[1]
            out[op] = solve(interior_except(ext, c), c, s1)
        elif op[1] == op[2]:
            c = op[1]
            out[op] = solve(interior_except(ext, c), c, s2)
        else:
            i, j = op[1], op[2]
            # D_j on rows extended along i, then D_i
            gj = solve(interior_except(ext, i + j), j, s1)
            a = solve(gj, i, s1)
            gi = solve(interior_except(ext, i + j), i, s1)
            b = solve(gi, j, s1)
            out[op] = (a + b) * 0.5
    return out


def apply_block(ext: np.ndarray, s1: Sch, s2: Sch, dx3: Sequence[float], N: int, g: int,
                ops: Iterable[str] = OPS) -> Dict[str, np.ndarray]:
    """Closed (no iteration) derivatives of one block with all ghosts filled."""
    res = apply_uniform(ext[None, None, None], s1, s2, dx3, N, g, ops, 0)
    return {k: v[0, 0, 0] for k, v in res.items()}


def laplacian_uniform(ext: np.ndarray, s2: Sch, dx3, N: int, g: int, n_iter: int = 0) -> np.ndarray:
    """sum_i D^{(2)}_i on the uniform decomposition (dxx + dyy + dzz)."""
    r = apply_uniform(ext, s2, s2, dx3, N, g, ("dxx", "dyy", "dzz"), n_iter)
    return r["dxx"] + r["dyy"] + r["dzz"]


def blocks_to_global(b: np.ndarray) -> np.ndarray:
    """(nbz, nby, nbx, N, N, N) interior blocks -> global (z, y, x) array."""
    nbz, nby, nbx, n0, n1, n2 = b.shape
    return b.transpose(0, 3, 1, 4, 2, 5).reshape(nbz * n0, nby * n1, nbx * n2)


def global_to_blocks(fg: np.ndarray, N: int) -> np.ndarray:
    nz, ny, nx = fg.shape
    return fg.reshape(nz // N, N, ny // N, N, nx // N, N).transpose(0, 2, 4, 1, 3, 5)


# ---------------------------------------------------------------------------
# Linear wave equation u_tt = Laplacian u with classical RK4
# ---------------------------------------------------------------------------


def wave_rhs(phi: np.ndarray, K: np.ndarray, s2: Sch, dx3, N: int, g: int, n_iter: int = 0):
    """Semi-discrete wave system with zero shift (Eq. toyShiftWaveEqnSys, beta = 0).

    d/dt Phi = K, d/dt K = sum_i D^{(2)}_i Phi.  ``phi`` and ``K`` are global
    periodic (z, y, x) arrays; the Laplacian is the decomposed operator.
    """
    lap = laplacian_uniform(ghost_fill_3d(phi, N, g), s2, dx3, N, g, n_iter)
    return K.copy(), blocks_to_global(lap)


def wave_rk4_step(phi: np.ndarray, K: np.ndarray, dt: float, s2: Sch, dx3, N: int, g: int,
                  n_iter: int = 0):
    """One classical ERK4 step (Sec. "Two dimensional advection", fully discrete)."""
    k1p, k1k = wave_rhs(phi, K, s2, dx3, N, g, n_iter)
    k2p, k2k = wave_rhs(phi + 0.5 * dt * k1p, K + 0.5 * dt * k1k, s2, dx3, N, g, n_iter)
    k3p, k3k = wave_rhs(phi + 0.5 * dt * k2p, K + 0.5 * dt * k2k, s2, dx3, N, g, n_iter)
    k4p, k4k = wave_rhs(phi + dt * k3p, K + dt * k3k, s2, dx3, N, g, n_iter)
    phi_n = phi + dt / 6.0 * (k1p + 2.0 * k2p + 2.0 * k3p + k4p)
    K_n = K + dt / 6.0 * (k1k + 2.0 * k2k + 2.0 * k3k + k4k)
    return phi_n, K_n
