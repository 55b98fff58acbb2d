"""Seeded synthetic inputs for the submatrix method (inputs only, no method arithmetic).

Shared by the oracle's tests, the GPU parity tests and ``bench.py``.  Nothing here
computes a submatrix, an inverse root or anything else of the method; it only builds
sparse symmetric matrices in CSR form (int32 ``rowptr``/``colind``, float64 ``vals``)
and random arrays of the shapes the method consumes.

The paper's own inputs (MATLAB ``sprandsym`` matrices, DFT overlap matrices,
SuiteSparse matrices; Sec. 4.1, 4.3, 4.4) are not available, so Gaussian-overlap
matrices stand in for them: points in a 3-D box, ``A_ij = exp(-r_ij^2 / 0.01)`` for
``r_ij < r_c`` (the sparsity of an overlap matrix of localised basis functions, the
paper's motivating application in Sec. 4.3), plus a diagonal that sets the condition
number.

Recipes (numpy PCG64, seed 0 unless stated):

* ``overlap_small``  n=2000 points U[0,1]^3, r_c=0.12, diagonal 1.5 (p=2, FP64).
* ``overlap_uniform`` n=32768 points U[0,L]^3 with L=1.0585 (about 177 stored
  entries per row), diagonal shift giving kappa(A) ~ 1e3.
* ``overlap_clustered`` n=131072 points in a periodic box of side 2: 85 % drawn from
  64 isotropic Gaussian clusters (std 0.1), 15 % uniform; minimum-image distances;
  kappa ~ 1e3.  Row sizes range 7..1113.
* ``overlap_grad`` n=16384 points U[0,0.9247]^3 (about 130 entries per row), kappa ~ 1e3.
* ``block_overlap`` 20000 atoms U[0,1]^3 (periodic) with 13 s-type Gaussian functions
  each (n = 260000): dense 13 x 13 blocks between atoms closer than the cutoff
  r_c = (64 / (20000 * 4/3 pi))^(1/3) (65 neighbour atoms including the atom itself);
  block entries are the overlaps of normalised Gaussians with exponents geometric in
  0.5 .. 8 r_c^-2, (2 sqrt(a b) / (a + b))^(3/2) exp(-a b / (a + b) r^2); diagonal shift
  to kappa ~ 1e4.  Submatrix orders are 13 x (number of neighbour atoms), ~845 on average.
* ``laplace2d_aniso``, ``jump3d`` (inputs of the preconditioning experiment, Sec. 4.4, whose
  SuiteSparse matrices are not available): an anisotropic 2-D 5-point Laplacian (64^2,
  coupling 1 / 0.01) and a 3-D 7-point operator with block-wise coefficients spanning four
  decades (16^3); both SPD, n = 4096.

Every generator can also be scaled down (``n=``) for fast tests; the box side is then
rescaled so the expected number of neighbours stays the same.
"""
from __future__ import annotations

import dataclasses
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla
import scipy.spatial

GAUSS_WIDTH = 0.01      # A_ij = exp(-r^2 / GAUSS_WIDTH)
CUTOFF = 0.12           # r_c


@dataclasses.dataclass
class CSR:
    """A sparse symmetric matrix in CSR form (sorted, unique column indices)."""
    n: int
    rowptr: np.ndarray      # int32 [n+1]
    colind: np.ndarray      # int32 [nnz]
    vals: np.ndarray        # float64 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.colind.shape[0])

    def row_sizes(self) -> np.ndarray:
        return np.diff(self.rowptr).astype(np.int64)

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.vals, self.colind, self.rowptr), shape=(self.n, self.n))


def _from_pairs(n, pairs, offvals, diag, name) -> CSR:
    i = np.concatenate([pairs[:, 0], pairs[:, 1], np.arange(n)])
    j = np.concatenate([pairs[:, 1], pairs[:, 0], np.arange(n)])
    v = np.concatenate([offvals, offvals, np.full(n, float(diag))])
    m = sp.csr_matrix((v, (i, j)), shape=(n, n))
    m.sum_duplicates()
    m.sort_indices()
    return CSR(n, m.indptr.astype(np.int32), m.indices.astype(np.int32),
               m.data.astype(np.float64), name)


def _pairs(points, cutoff, box=None):
    tree = scipy.spatial.cKDTree(points, boxsize=box)
    pairs = tree.query_pairs(cutoff, output_type="ndarray").astype(np.int64)
    d = points[pairs[:, 0]] - points[pairs[:, 1]]
    if box is not None:
        d -= box * np.round(d / box)
    r2 = (d * d).sum(1)
    return pairs, np.exp(-r2 / GAUSS_WIDTH)


def _row_split_operator(m: sp.csr_matrix):
    """x -> m x as a LinearOperator whose product runs over row blocks in threads.  Each
    row's sum is formed exactly as in ``m @ x``, so the result (and every Lanczos run built
    on it) is bit-identical to the single-threaded product."""
    n = m.shape[0]
    k = max(1, min(16, os.cpu_count() or 1, n // 4096))
    bounds = np.linspace(0, n, k + 1).astype(np.int64)
    parts = [m[bounds[i]:bounds[i + 1]] for i in range(k)]
    pool = ThreadPoolExecutor(k)

    def mv(x):
        x = np.asarray(x, dtype=np.float64).ravel()
        return np.concatenate(list(pool.map(lambda part: part @ x, parts)))

    return sla.LinearOperator((n, n), matvec=mv, dtype=np.float64), pool


def _extreme_eig_pair(m: sp.csr_matrix, seed: int):
    """Largest and smallest eigenvalue of the symmetric m (ARPACK Lanczos, seeded start);
    the smallest via the largest of (hi I - m), which Lanczos separates better."""
    v0 = np.random.default_rng(seed).standard_normal(m.shape[0])
    op, pool = _row_split_operator(m)
    hi = sla.eigsh(op, k=1, which="LA", v0=v0, tol=1e-8, return_eigenvectors=False)[0]
    pool.shutdown()
    op, pool = _row_split_operator((hi * sp.identity(m.shape[0], format="csr") - m).tocsr())
    lo = hi - sla.eigsh(op, k=1, which="LA", v0=v0, tol=1e-8, return_eigenvectors=False)[0]
    pool.shutdown()
    return float(lo), float(hi)


def _extreme_eigs(n, pairs, offvals, seed=0):
    """Extreme eigenvalues of the zero-diagonal part (ARPACK Lanczos, seeded start)."""
    i = np.concatenate([pairs[:, 0], pairs[:, 1]])
    j = np.concatenate([pairs[:, 1], pairs[:, 0]])
    off = sp.csr_matrix((np.concatenate([offvals, offvals]), (i, j)), shape=(n, n))
    return _extreme_eig_pair(off, seed)


def diag_for_kappa(lo: float, hi: float, kappa: float) -> float:
    """Diagonal value d with (hi + d) / (lo + d) = kappa."""
    return (hi - kappa * lo) / (kappa - 1.0)


def overlap_small(n: int = 2000, seed: int = 0, diag: float = 1.5) -> CSR:
    """n points U[0,1]^3 (non-periodic), r_c = 0.12, literal diagonal 1 + 0.5."""
    rng = np.random.default_rng(seed)
    side = (n / 2000.0) ** (1.0 / 3.0)
    pts = rng.uniform(0.0, side, (n, 3))
    pairs, v = _pairs(pts, CUTOFF)
    return _from_pairs(n, pairs, v, diag, f"overlap_small(n={n})")


def _uniform_side(n, per_row):
    # expected neighbours inside the cutoff ball = n / L^3 * 4/3 pi r_c^3
    return (n * (4.0 / 3.0) * np.pi * CUTOFF ** 3 / per_row) ** (1.0 / 3.0)


def overlap_uniform(n: int = 32768, seed: int = 0, kappa: float = 1e3,
                    per_row: float = 200.0, side: float | None = None) -> CSR:
    """Uniform points in a cube sized for about ``per_row`` neighbours; kappa via the diagonal."""
    rng = np.random.default_rng(seed)
    if side is None:
        side = _uniform_side(n, per_row)
    pts = rng.uniform(0.0, side, (n, 3))
    pairs, v = _pairs(pts, CUTOFF)
    lo, hi = _extreme_eigs(n, pairs, v, seed)
    d = diag_for_kappa(lo, hi, kappa)
    return _from_pairs(n, pairs, v, d, f"overlap_uniform(n={n},kappa={kappa:g})")


def overlap_grad(n: int = 16384, seed: int = 0, kappa: float = 1e3) -> CSR:
    """The differentiation workload: n=16384 in U[0,0.9247]^3 (about 130 per row)."""
    side = 0.9247 * (n / 16384.0) ** (1.0 / 3.0)
    return overlap_uniform(n, seed, kappa, side=side)


def overlap_clustered(n: int = 131072, seed: int = 0, kappa: float = 1e3,
                      clusters: int = 64, frac_clustered: float = 0.85) -> CSR:
    """Gaussian-mixture points in a periodic box: uneven row sizes (7..1113 at n=131072)."""
    rng = np.random.default_rng(seed)
    side = 2.0 * (n / 131072.0) ** (1.0 / 3.0)
    nc = int(frac_clustered * n)
    centres = rng.uniform(0.0, side, (clusters, 3))
    labels = rng.integers(0, clusters, nc)
    pts = np.concatenate([centres[labels] + rng.normal(0.0, 0.05 * side, (nc, 3)),
                          rng.uniform(0.0, side, (n - nc, 3))]) % side
    pairs, v = _pairs(pts, CUTOFF, box=side)
    lo, hi = _extreme_eigs(n, pairs, v, seed)
    d = diag_for_kappa(lo, hi, kappa)
    return _from_pairs(n, pairs, v, d, f"overlap_clustered(n={n},kappa={kappa:g})")


def random_sparse_spd(n: int, density: float, seed: int = 0, margin: float = 0.5) -> CSR:
    """Small random symmetric sparse matrix made SPD by diagonal dominance plus ``margin``.

    Used for brute-force and edge-case tests (tiny n)."""
    rng = np.random.default_rng(seed)
    mask = np.triu(rng.random((n, n)) < density, 1)
    vals = rng.uniform(-1.0, 1.0, (n, n)) * mask
    dense = vals + vals.T
    dense += np.diag(np.abs(dense).sum(1) + margin)
    return dense_to_csr(dense, f"random_sparse_spd(n={n})")


def dense_to_csr(dense: np.ndarray, name: str = "", keep=None) -> CSR:
    """CSR of a dense matrix; the stored pattern is ``keep`` (default: nonzeros + diagonal)."""
    n = dense.shape[0]
    if keep is None:
        keep = (dense != 0) | np.eye(n, dtype=bool)
    # store explicit zeros that ``keep`` asks for
    r, c = np.nonzero(keep)
    m = sp.csr_matrix((dense[r, c], (r, c)), shape=(n, n))
    m.sort_indices()
    return CSR(n, m.indptr.astype(np.int32), m.indices.astype(np.int32),
               m.data.astype(np.float64), name)


def random_on_pattern(a: CSR, seed: int, symmetric: bool = False) -> np.ndarray:
    """N(0,1) values on A's pattern (length nnz); optionally symmetrised (E_rc = E_cr)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(a.nnz)
    if symmetric:
        m = sp.csr_matrix((w, a.colind, a.rowptr), shape=(a.n, a.n))
        m = (m + m.T) * 0.5
        m = m.tocsr()
        m.sort_indices()
        # same pattern (A's pattern is symmetric), so data lines up with colind
        assert m.nnz == a.nnz and np.array_equal(m.indices, a.colind)
        w = m.data.copy()
    return w


def block_diagonal_spd(blocks: int, size: int, seed: int = 0) -> CSR:
    """``blocks`` dense random SPD blocks of one order ``size`` on the diagonal, each stored in
    full, so every row's submatrix has order exactly ``size`` (Q Q^T / size + 0.5 I with Q
    standard normal, numpy PCG64).  Used to time the engines per row size."""
    rng = np.random.default_rng(seed)
    n = blocks * size
    qs = rng.standard_normal((blocks, size, size))
    vals = np.einsum("bij,bkj->bik", qs, qs) / size + 0.5 * np.eye(size)[None]
    r = np.arange(n, dtype=np.int64)
    blk = r // size
    rowptr = (np.arange(n + 1, dtype=np.int64) * size).astype(np.int32)
    colind = (blk[:, None] * size + np.arange(size)[None, :]).ravel().astype(np.int32)
    v = vals[blk, r % size, :].ravel().astype(np.float64)
    return CSR(n, rowptr, colind, v, f"block_diagonal_spd(blocks={blocks},size={size})")


def stratified_rows(m: np.ndarray, k: int, seed: int = 3) -> np.ndarray:
    """A seeded sample of about k row indices stratified by row size: the sizes are binned
    by powers of two (below 32, 32..63, ..., 1024..2047, 2048 and above), each non-empty bin
    gives an equal share (all its rows if it has fewer), and the rows of the smallest and
    the largest size are always included.  Sorted, unique."""
    m = np.asarray(m)
    rng = np.random.default_rng(seed)
    edges = [0, 32, 64, 128, 256, 512, 1024, 2048, np.iinfo(np.int64).max]
    bins = [np.nonzero((m >= lo) & (m < hi))[0] for lo, hi in zip(edges[:-1], edges[1:])]
    bins = [b for b in bins if len(b)]
    share = max(1, k // max(1, len(bins)))
    pick = [np.nonzero(m == m.min())[0][:1], np.nonzero(m == m.max())[0][:1]]
    for b in bins:
        pick.append(b if len(b) <= share else rng.choice(b, size=share, replace=False))
    return np.unique(np.concatenate(pick)).astype(np.int64)


def block_overlap(atoms: int = 20000, funcs: int = 13, seed: int = 0,
                  kappa: float = 1e4) -> CSR:
    """Block-sparse Gaussian-basis overlap matrix (n = atoms * funcs), see the module doc."""
    rng = np.random.default_rng(seed)
    rc = (64.0 / (20000 * 4.0 / 3.0 * np.pi)) ** (1.0 / 3.0)
    side = (atoms / 20000.0) ** (1.0 / 3.0)            # same atom density at any size
    pos = rng.uniform(0.0, side, (atoms, 3))
    tree = scipy.spatial.cKDTree(pos, boxsize=side)
    pairs = tree.query_pairs(rc, output_type="ndarray").astype(np.int64)
    d = pos[pairs[:, 0]] - pos[pairs[:, 1]]
    d -= side * np.round(d / side)
    r2 = (d * d).sum(1)
    alpha = 0.5 * 16.0 ** (np.arange(funcs) / (funcs - 1)) / rc ** 2
    prod = alpha[:, None] * alpha[None, :]
    tot = alpha[:, None] + alpha[None, :]
    pref = (2.0 * np.sqrt(prod) / tot) ** 1.5
    red = prod / tot
    f = np.arange(funcs)
    # off-diagonal blocks (a < b) and their transposes, then the diagonal blocks (r = 0)
    blk = pref[None] * np.exp(-red[None] * r2[:, None, None])
    ia = (pairs[:, 0, None, None] * funcs + f[None, :, None]) + 0 * f[None, None, :]
    jb = (pairs[:, 1, None, None] * funcs + f[None, None, :]) + 0 * f[None, :, None]
    ad = np.arange(atoms)
    id_ = (ad[:, None, None] * funcs + f[None, :, None]) + 0 * f[None, None, :]
    jd_ = (ad[:, None, None] * funcs + f[None, None, :]) + 0 * f[None, :, None]
    n = atoms * funcs
    i = np.concatenate([ia.ravel(), jb.ravel(), id_.ravel()])
    j = np.concatenate([jb.ravel(), ia.ravel(), jd_.ravel()])
    v = np.concatenate([blk.ravel(), blk.ravel(), np.broadcast_to(pref, (atoms, funcs, funcs)).ravel()])
    g = sp.csr_matrix((v, (i, j)), shape=(n, n))
    g.sum_duplicates()
    lo, hi = _extreme_eig_pair(g, seed)
    g = (g + diag_for_kappa(lo, hi, kappa) * sp.identity(n, format="csr")).tocsr()
    g.sort_indices()
    return CSR(n, g.indptr.astype(np.int32), g.indices.astype(np.int32),
               g.data.astype(np.float64), f"block_overlap(atoms={atoms},funcs={funcs},kappa={kappa:g})")


def _stencil_csr(offdiag: dict, diag: np.ndarray, name: str) -> CSR:
    """CSR of a symmetric matrix from its off-diagonal pairs {(i, j): v} (i < j) and its
    diagonal."""
    n = diag.shape[0]
    if offdiag:
        ij = np.array(list(offdiag.keys()), dtype=np.int64)
        v = np.array(list(offdiag.values()), dtype=np.float64)
    else:
        ij = np.zeros((0, 2), dtype=np.int64)
        v = np.zeros(0)
    return _from_pairs_diag(n, ij, v, diag, name)


def _from_pairs_diag(n, pairs, offvals, diag, name) -> CSR:
    i = np.concatenate([pairs[:, 0], pairs[:, 1], np.arange(n)])
    j = np.concatenate([pairs[:, 1], pairs[:, 0], np.arange(n)])
    v = np.concatenate([offvals, offvals, diag])
    m = sp.csr_matrix((v, (i, j)), shape=(n, n))
    m.sum_duplicates()
    m.sort_indices()
    return CSR(n, m.indptr.astype(np.int32), m.indices.astype(np.int32),
               m.data.astype(np.float64), name)


def laplace2d_aniso(nx: int = 64, eps: float = 0.01) -> CSR:
    """Stand-in for the SuiteSparse SPD matrices of the preconditioning experiment
    (Sec. 4.4, 1000 <= n <= 5000, not available here): the 5-point Dirichlet Laplacian on an
    nx x nx grid with coupling 1 along x and eps along y (n = nx^2; condition number
    ~ 4 / ((1 + eps) (pi / (nx + 1))^2), ~1.7e3 at the defaults)."""
    n = nx * nx
    off = {}
    diag = np.zeros(n)
    for y in range(nx):
        for x in range(nx):
            k = y * nx + x
            diag[k] = 2.0 + 2.0 * eps
            if x + 1 < nx:
                off[(k, k + 1)] = -1.0
            if y + 1 < nx:
                off[(k, k + nx)] = -eps
    return _stencil_csr(off, diag, f"laplace2d_aniso(nx={nx},eps={eps:g})")


def jump3d(nx: int = 16, contrast: float = 1e4, seed: int = 0) -> CSR:
    """Second stand-in for Sec. 4.4: the 7-point finite-volume operator of -div(c grad u)
    on an nx^3 grid (Dirichlet), with c piecewise constant on 4^3-cell blocks, each block's
    c = contrast^u, u ~ U[0,1] (numpy PCG64, seed); face coefficients are harmonic means.
    n = nx^3 (4096 at the defaults)."""
    rng = np.random.default_rng(seed)
    nb = (nx + 3) // 4
    cb = contrast ** rng.random((nb, nb, nb))
    c = cb[np.arange(nx)[:, None, None] // 4, np.arange(nx)[None, :, None] // 4,
           np.arange(nx)[None, None, :] // 4]
    n = nx ** 3
    idx = np.arange(n).reshape(nx, nx, nx)
    off = {}
    diag = np.zeros(n)
    for axis in range(3):
        a = np.moveaxis(c, axis, 0)
        ia = np.moveaxis(idx, axis, 0)
        h = 2.0 * a[:-1] * a[1:] / (a[:-1] + a[1:])           # interior faces
        for k0, k1, w in zip(ia[:-1].ravel(), ia[1:].ravel(), h.ravel()):
            off[(int(min(k0, k1)), int(max(k0, k1)))] = -float(w)
            diag[k0] += w
            diag[k1] += w
        diag[ia[0].ravel()] += 2.0 * a[0].ravel()            # Dirichlet boundary faces
        diag[ia[-1].ravel()] += 2.0 * a[-1].ravel()
    return _stencil_csr(off, diag, f"jump3d(nx={nx},contrast={contrast:g},seed={seed})")


WORKLOADS = {
    "overlap_small": overlap_small,
    "overlap_uniform": overlap_uniform,
    "overlap_clustered": overlap_clustered,
    "overlap_grad": overlap_grad,
    "block_overlap": block_overlap,
    "laplace2d_aniso": laplace2d_aniso,
    "jump3d": jump3d,
}
