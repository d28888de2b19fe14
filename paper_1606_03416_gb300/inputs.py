"""Seeded synthetic inputs for DG-CheFSI: block-sparse H, starting block X, Lanczos start vector.

This module builds inputs only. It holds none of the method's arithmetic
(no mat-vec, no filter, no orthonormalisation, no eigensolve of H), so the
FP64 oracle and the CUDA path can both be fed from it without sharing code.

Structure being imitated (paper Sec. II.B, Eq. HDG_sub_blocks and Fig. 1):
H is symmetric, partitioned into element blocks H_{K;K'} of size J_K x J_K',
and a block is nonzero only when elements K and K' are neighbours. The paper's
own Hamiltonians (DFT on Li-ion electrolyte and graphene) are not available, so
blocks are drawn at random with a spectrum of the right kind:

* diagonal block  H_KK  = Q diag(d) Q^T,  d ~ U[-1, 40],  Q Haar-orthogonal
  (QR of a Gaussian matrix with the signs of diag(R) made positive), then
  symmetrised exactly as (H + H^T)/2;
* off-diagonal pair {K < K'}: B = s * Gaussian(n_K x n_K'), H_KK' = B,
  H_K'K = B^T, with s set by the neighbour class of the offset
  (1 = face, 2 = edge, 3 = corner in 3D; 1 = side, 2 = diagonal in 2D).

Draw order from ``numpy.random.default_rng(seed)`` (fixed, so a seed fixes the
problem): the per-element sizes (only when uneven) -> diagonal blocks in element
order (G then d) -> off-diagonal pairs in lexicographic (K, K') order. The
starting block X and the Lanczos start vector come from their own generators
(seeds ``seed + 1`` and ``seed + 2``) so the matrix does not depend on N_s.

Layout returned (the library's layout as well):
* block-CSR over elements: ``row_ptr[M+1]`` (int64), ``col[nnzb]`` (int32,
  ascending per row, every row holds its diagonal), ``blk_off[nnzb]`` (int64,
  offset in doubles into ``values``), ``values`` (float64, each block row-major
  n_K x n_K');
* X as a (N_s, N) C-contiguous float64 array: row i is state i, so the paper's
  N x N_s block of column vectors is ``X.T``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import itertools
import math

import numpy as np


@dataclass(frozen=True)
class ProblemConfig:
    """One synthetic DG-CheFSI workload.

    grid      elements per axis (gx, gy, gz); element K = x + gx*(y + gy*z)
    periodic  wrap-around per axis
    stencil   "27" (3D, offsets in {-1,0,1}^3) or "9" (2D, {-1,0,1}^2 x {0})
    nb        basis functions per element: an int, or (lo, hi) for U{lo..hi}
    Ns        number of states (columns of X)
    m         Chebyshev filter degree
    Ne        electron count (2 per fully occupied state: spin factor)
    kT        Fermi-Dirac smearing, same units as H
    scales    off-diagonal scale per neighbour class
    """

    name: str
    grid: tuple
    periodic: tuple
    stencil: str
    nb: object
    Ns: int
    m: int
    Ne: float
    kT: float = 0.01
    scales: dict = field(default_factory=lambda: {1: 0.05, 2: 0.02, 3: 0.01})
    seed: int = 0
    cycles: int = 1

    @property
    def M(self) -> int:
        return int(np.prod(self.grid))


def default_ne(Ns: int) -> float:
    """Electron count when the workload does not state one: leave
    max(16, ceil(0.03 Ns)) states empty above the occupied ones (the paper adds
    100-120 spare states to a few thousand occupied ones, Sec. IV)."""
    return float(2 * (Ns - max(16, math.ceil(0.03 * Ns))))


# The workloads. Sizes are those of the five DG-CheFSI benchmark settings:
# a tiny all-coupled 2x2x2 problem, a bulk-3D-like 8^3 grid, a graphene-like
# 2D sheet with uneven element sizes, and a 12^3 grid for differentiation.
CONFIGS = {
    "tiny_2x2x2": ProblemConfig(
        name="tiny_2x2x2", grid=(2, 2, 2), periodic=(True, True, True), stencil="27",
        nb=32, Ns=48, m=10, Ne=64.0, kT=0.01,
        scales={1: 0.05, 2: 0.05, 3: 0.05}, seed=0, cycles=20),
    "bulk3d_8x8x8": ProblemConfig(
        name="bulk3d_8x8x8", grid=(8, 8, 8), periodic=(True, True, True), stencil="27",
        nb=64, Ns=4096, m=20, Ne=default_ne(4096), kT=0.01,
        scales={1: 0.05, 2: 0.02, 3: 0.01}, seed=0),
    "sheet2d_24x20": ProblemConfig(
        name="sheet2d_24x20", grid=(24, 20, 1), periodic=(True, True, False), stencil="9",
        nb=(40, 120), Ns=-1, m=16, Ne=-1.0, kT=0.01,
        scales={1: 0.05, 2: 0.02}, seed=0),
    "bulk3d_12x12x12": ProblemConfig(
        name="bulk3d_12x12x12", grid=(12, 12, 12), periodic=(True, True, True), stencil="27",
        nb=48, Ns=8192, m=24, Ne=default_ne(8192), kT=0.01,
        scales={1: 0.05, 2: 0.02, 3: 0.01}, seed=0),
}


def scaled_copy(cfg: ProblemConfig, grid=None, nb=None, Ns=None, m=None, Ne=None, name=None) -> ProblemConfig:
    """A smaller copy of a workload: same generator and stencil, other sizes."""
    g = tuple(grid) if grid is not None else cfg.grid
    ns = Ns if Ns is not None else cfg.Ns
    return ProblemConfig(
        name=name or f"{cfg.name}_copy", grid=g, periodic=cfg.periodic, stencil=cfg.stencil,
        nb=nb if nb is not None else cfg.nb, Ns=ns, m=m if m is not None else cfg.m,
        Ne=Ne if Ne is not None else default_ne(ns), kT=cfg.kT, scales=dict(cfg.scales),
        seed=cfg.seed, cycles=cfg.cycles)


def _offsets(stencil: str):
    if stencil == "27":
        return [o for o in itertools.product((-1, 0, 1), repeat=3) if o != (0, 0, 0)]
    if stencil == "9":
        return [(dx, dy, 0) for dx, dy in itertools.product((-1, 0, 1), repeat=2) if (dx, dy) != (0, 0)]
    raise ValueError(f"unknown stencil {stencil!r}")


def neighbour_classes(cfg: ProblemConfig):
    """For each element K: dict K' -> neighbour class (number of nonzero offset
    components; the smallest one when several offsets reach the same K')."""
    gx, gy, gz = cfg.grid
    out = []
    for K in range(cfg.M):
        x, y, z = K % gx, (K // gx) % gy, K // (gx * gy)
        nbrs = {}
        for off in _offsets(cfg.stencil):
            c = [x + off[0], y + off[1], z + off[2]]
            ok = True
            for ax, n in enumerate((gx, gy, gz)):
                if cfg.periodic[ax]:
                    c[ax] %= n
                elif not 0 <= c[ax] < n:
                    ok = False
            if not ok:
                continue
            Kp = c[0] + gx * (c[1] + gy * c[2])
            if Kp == K:
                continue
            cls = sum(1 for o in off if o != 0)
            nbrs[Kp] = min(cls, nbrs.get(Kp, 99))
        out.append(nbrs)
    return out


@dataclass
class BlockSparse:
    """Host copy of a symmetric block-sparse H in block-CSR form."""
    nb: np.ndarray        # int32 [M]
    row_ptr: np.ndarray   # int64 [M+1]
    col: np.ndarray       # int32 [nnzb]
    blk_off: np.ndarray   # int64 [nnzb]
    values: np.ndarray    # float64 [sum of block sizes]

    @property
    def M(self) -> int:
        return int(self.nb.shape[0])

    @property
    def N(self) -> int:
        return int(self.nb.sum())

    @property
    def nnzb(self) -> int:
        return int(self.col.shape[0])


def make_blocks(cfg: ProblemConfig) -> BlockSparse:
    rng = np.random.default_rng(cfg.seed)
    M = cfg.M
    if isinstance(cfg.nb, tuple):
        lo, hi = cfg.nb
        nb = rng.integers(lo, hi + 1, size=M).astype(np.int32)
    else:
        nb = np.full(M, int(cfg.nb), dtype=np.int32)
    diag = []
    for K in range(M):
        n = int(nb[K])
        G = rng.standard_normal((n, n))
        d = rng.uniform(-1.0, 40.0, size=n)
        Q, R = np.linalg.qr(G)
        Q = Q * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]
        Hk = (Q * d[None, :]) @ Q.T
        diag.append(0.5 * (Hk + Hk.T))
    classes = neighbour_classes(cfg)
    off = {}
    for K in range(M):
        for Kp in sorted(classes[K]):
            if Kp > K:
                s = cfg.scales[classes[K][Kp]]
                off[(K, Kp)] = s * rng.standard_normal((int(nb[K]), int(nb[Kp])))
    row_ptr = np.zeros(M + 1, dtype=np.int64)
    cols, offs, vals = [], [], []
    pos = 0
    for K in range(M):
        row = sorted(set(classes[K]) | {K})
        for Kp in row:
            if Kp == K:
                blk = diag[K]
            elif Kp > K:
                blk = off[(K, Kp)]
            else:
                blk = off[(Kp, K)].T
            cols.append(Kp)
            offs.append(pos)
            vals.append(np.ascontiguousarray(blk).ravel())
            pos += blk.size
        row_ptr[K + 1] = len(cols)
    return BlockSparse(nb=nb, row_ptr=row_ptr, col=np.asarray(cols, dtype=np.int32),
                       blk_off=np.asarray(offs, dtype=np.int64),
                       values=np.concatenate(vals).astype(np.float64))


def resolve_sizes(cfg: ProblemConfig, H: BlockSparse):
    """N_s and N_e for workloads that state them relative to N (the 2D sheet:
    N_s = floor(0.55 N))."""
    Ns = cfg.Ns if cfg.Ns > 0 else int(math.floor(0.55 * H.N))
    Ne = cfg.Ne if cfg.Ne >= 0 else default_ne(Ns)
    return Ns, Ne


def make_X(N: int, Ns: int, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """Random Gaussian starting block, (N_s, N) C-contiguous (row i = state i)."""
    rng = np.random.default_rng(seed + 1)
    return rng.standard_normal((Ns, N), dtype=np.float64).astype(dtype, copy=False)


def make_start_vector(N: int, seed: int = 0) -> np.ndarray:
    """Gaussian start vector for the Lanczos bound (not normalised)."""
    rng = np.random.default_rng(seed + 2)
    return rng.standard_normal(N)


def make_problem(cfg: ProblemConfig):
    """(H, X0, v0, Ns, Ne) for a workload."""
    H = make_blocks(cfg)
    Ns, Ne = resolve_sizes(cfg, H)
    return H, make_X(H.N, Ns, cfg.seed), make_start_vector(H.N, cfg.seed), Ns, Ne


def _orthonormal_columns(rng, R: int, n: int) -> np.ndarray:
    """R x n with orthonormal columns (QR of a Gaussian, signs fixed)."""
    Q, Rf = np.linalg.qr(rng.standard_normal((R, n)))
    return Q * np.where(np.diag(Rf) < 0, -1.0, 1.0)[None, :]


def make_basis_pair(nb_old, nb_new, nr, delta: float = 0.05, seed: int = 0):
    """Synthetic adaptive local bases of two consecutive SCF steps, sampled on
    each element's grid points: per element K an R_K x J_K^{old} matrix with
    orthonormal columns, and an R_K x J_K^{new} one spanning a perturbation of
    it (the old columns plus delta-scaled Gaussian noise, extended by random
    directions when the element gains basis functions), the kind of small basis
    change between SCF steps that re-alignment is for. Returns
    (V_old list, V_new list)."""
    rng = np.random.default_rng(seed + 3)
    V_old, V_new = [], []
    for K in range(len(nb_old)):
        R, n0, n1 = int(nr[K]), int(nb_old[K]), int(nb_new[K])
        if not (1 <= n0 <= R and 1 <= n1 <= R):
            raise ValueError("need 1 <= basis functions <= grid points on every element")
        A = _orthonormal_columns(rng, R, n0)
        B = np.hstack([A, rng.standard_normal((R, max(n1 - n0, 0)))])[:, :n1]
        Q, Rf = np.linalg.qr(B + delta * rng.standard_normal((R, n1)))
        V_old.append(A)
        V_new.append(Q * np.where(np.diag(Rf) < 0, -1.0, 1.0)[None, :])
    return V_old, V_new


def make_planted_symmetric(lam, seed: int = 0) -> np.ndarray:
    """A symmetric n x n matrix Q diag(lam) Q^T with Q Haar-orthogonal (QR of a
    Gaussian, signs fixed), symmetrised exactly as (A + A^T)/2: a stand-in for a
    projected Hamiltonian with a chosen spectrum (clusters, repeated values)."""
    lam = np.asarray(lam, dtype=np.float64)
    rng = np.random.default_rng(seed + 4)
    Q = _orthonormal_columns(rng, lam.size, lam.size)
    A = (Q * lam[None, :]) @ Q.T
    return 0.5 * (A + A.T)


def clustered_spectrum(n: int, groups=(), lo: float = -1.3, hi: float = 2.0, seed: int = 0) -> np.ndarray:
    """n ascending values: n - sum(sizes) uniform on [lo, hi] plus, for each
    (centre, size, spread) in groups, `size` values centre + spread * Gaussian
    (spread 0: a value repeated `size` times)."""
    rng = np.random.default_rng(seed + 5)
    parts = [rng.uniform(lo, hi, n - sum(g[1] for g in groups))]
    for centre, size, spread in groups:
        parts.append(centre + spread * rng.standard_normal(size))
    return np.sort(np.concatenate(parts))


def near_diagonal_symmetric(d, coupling: float, top: int = 0, top_coupling: float = 0.0, seed: int = 0) -> np.ndarray:
    """diag(d) plus a symmetric Gaussian perturbation of size `coupling`, and
    of size `top_coupling` among the last `top` rows and columns: the shape of
    a projected Hamiltonian in the basis of a converging subspace iteration
    (converged states nearly decoupled, the unconverged top block not)."""
    d = np.asarray(d, dtype=np.float64)
    n = d.size
    rng = np.random.default_rng(seed + 6)
    P = coupling * rng.standard_normal((n, n))
    if top > 0:
        P[n - top:, n - top:] = top_coupling * rng.standard_normal((top, top))
    A = np.diag(d) + 0.5 * (P + P.T)
    return 0.5 * (A + A.T)


def planted_cholesky(n: int, cond: float = 1e3, negative_at: int = -1, seed: int = 0):
    """(S, L): S = L D L^T with L lower triangular, unit-scale Gaussian below
    the diagonal and a positive diagonal spread log-uniformly over [1, sqrt(cond)],
    D = I except D[negative_at] = -1 (then S is indefinite and its Cholesky
    factorisation meets its first non-positive pivot at that row). S is
    symmetrised exactly."""
    rng = np.random.default_rng(seed + 7)
    L = np.tril(rng.standard_normal((n, n)), -1) / np.sqrt(max(n, 1))
    L[np.diag_indices(n)] = np.exp(rng.uniform(0.0, 0.5 * np.log(cond), n))
    d = np.ones(n)
    if negative_at >= 0:
        d[negative_at] = -1.0
    S = (L * d[None, :]) @ L.T
    return 0.5 * (S + S.T), L


def pack_blocks(blocks) -> np.ndarray:
    """Concatenate row-major blocks into one float64 array (the packed layout
    of the re-alignment call)."""
    return np.concatenate([np.ascontiguousarray(b, dtype=np.float64).ravel() for b in blocks])
