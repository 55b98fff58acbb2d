"""FP64 CPU oracle for the submatrix method (Lass et al., "A Massively Parallel
Algorithm for the Approximate Calculation of Inverse p-th Roots of Large Sparse
Matrices", PASC'18).

TEST INFRASTRUCTURE ONLY.  This module is plain, slow and meant to be obviously
correct; it shares no code with the CUDA library.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import it.  The product path never calls it.

What it computes, in the paper's order:

* Algorithm 1 (Sec. 3.1): for row/column j, the index set R = {i : A_ij stored}
  (ascending) and the dense principal submatrix S[k][l] = A[R[k]][R[l]].
* Sec. 3.2: the submatrix operation f(S) = S^(-1/p).  The paper leaves the solver
  open; for a symmetric matrix it names the route through the spectral
  decomposition (Sec. 2): S = V diag(lambda) V^T, f(S) = V diag(lambda^(-1/p)) V^T
  with the principal real root.  ``numpy.linalg.eigh`` (LAPACK) is that step.
* Algorithm 2 (Sec. 3.3) with the row-based storage of Sec. 3.4: row j of the CSR
  result holds column R.indexof(j) of f(S_j), in the order of R, i.e. the result
  reuses A's rowptr/colind and only the value array is new.
* Sec. 4.2 applies the same method to positive p-th roots; every function below takes
  ``sign=-1`` (the default, f(S) = S^(-1/p)) or ``sign=+1`` (f(S) = S^(1/p)).

Readings where the paper is silent (each also listed in the design notes):

* "nonzero" means *stored* in the pattern (an explicitly stored zero counts).
* The diagonal entry A_jj must be stored, otherwise R.indexof(j) is undefined; the
  oracle raises ``ValueError``.
* An indefinite submatrix has no principal real inverse root; the oracle raises.
* The gradient (``grad``) is with respect to the stored values of a symmetric A, with
  the (r,c)/(c,r) pair sharing one symmetric perturbation: the incoming column
  cotangent g of row j is symmetrised as (g e_pos^T + e_pos g^T)/2 before the
  Daleckii-Krein formula (Higham, Functions of Matrices, Thm. 3.11) is applied.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------------------
# Algorithm 1: index sets and dense submatrices
# ---------------------------------------------------------------------------

def index_set(rowptr, colind, j):
    """R_j: the stored column indices of row j (Alg. 1, collected in ascending order)."""
    return np.asarray(colind[rowptr[j]:rowptr[j + 1]], dtype=np.int64)


def plan(rowptr, colind):
    """Integer plan of Alg. 1/2: m_j = |R_j| and pos_j = R_j.indexof(j).

    Returns (m, pos) as int64 arrays.  Raises ``ValueError`` when a diagonal entry is
    not stored (Alg. 2 needs R.indexof(j))."""
    n = len(rowptr) - 1
    m = np.zeros(n, dtype=np.int64)
    pos = np.zeros(n, dtype=np.int64)
    for j in range(n):
        r = index_set(rowptr, colind, j)
        m[j] = len(r)
        hit = np.nonzero(r == j)[0]
        if len(hit) != 1:
            raise ValueError(f"row {j}: diagonal entry not stored")
        pos[j] = hit[0]
    return m, pos


def submatrix(rowptr, colind, vals, j):
    """Alg. 1 for one column: (S_j, R_j, pos_j) with S_j[k][l] = A[R[k]][R[l]]."""
    r = index_set(rowptr, colind, j)
    m = len(r)
    s = np.zeros((m, m), dtype=np.float64)
    for k in range(m):
        row = r[k]
        cols = np.asarray(colind[rowptr[row]:rowptr[row + 1]], dtype=np.int64)
        v = np.asarray(vals[rowptr[row]:rowptr[row + 1]], dtype=np.float64)
        # A[R[k]][R[l]] is the stored value of row R[k] at column R[l], else 0
        where = np.searchsorted(cols, r)
        ok = where < len(cols)
        ok[ok] &= cols[where[ok]] == r[ok]
        s[k, ok] = v[where[ok]]
    hit = np.nonzero(r == j)[0]
    if len(hit) != 1:
        raise ValueError(f"row {j}: diagonal entry not stored")
    return s, r, int(hit[0])


# ---------------------------------------------------------------------------
# Sec. 3.2: the submatrix operation
# ---------------------------------------------------------------------------

def inv_root(s, p, sign=-1):
    """S^(sign/p) of a symmetric positive definite S via its eigendecomposition."""
    lam, v = np.linalg.eigh(s)
    if lam[0] <= 0.0:
        raise ValueError(f"submatrix not positive definite (lambda_min = {lam[0]:.3e})")
    return (v * lam ** (sign / p)) @ v.T


def inv_root_column(s, pos, p, sign=-1):
    """Column pos of S^(sign/p) (the only column Alg. 2 keeps)."""
    lam, v = np.linalg.eigh(s)
    if lam[0] <= 0.0:
        raise ValueError(f"submatrix not positive definite (lambda_min = {lam[0]:.3e})")
    return v @ (lam ** (sign / p) * v[pos, :])


# ---------------------------------------------------------------------------
# Alg. 1 + Sec. 3.2 + Alg. 2: the whole method
# ---------------------------------------------------------------------------

def invroot(rowptr, colind, vals, p, rows=None, sign=-1):
    """The submatrix method's approximation of A^(sign/p) on A's CSR pattern.

    Returns the value array of the result (length nnz; same rowptr/colind as A).
    With ``rows`` given, only those rows' segments are computed and the rest of the
    returned array is NaN."""
    nnz = len(colind)
    out = np.full(nnz, np.nan)
    n = len(rowptr) - 1
    for j in (range(n) if rows is None else rows):
        s, r, pos = submatrix(rowptr, colind, vals, j)
        out[rowptr[j]:rowptr[j + 1]] = inv_root_column(s, pos, p, sign)
    return out


def row_segment(rowptr, colind, vals, p, j, sign=-1):
    """Row j of the result alone (column pos_j of S_j^(sign/p))."""
    s, r, pos = submatrix(rowptr, colind, vals, j)
    return inv_root_column(s, pos, p, sign)


# ---------------------------------------------------------------------------
# The paper's own p = 1 route (Sec. 6.1): LU factorisation and inversion per submatrix
# ---------------------------------------------------------------------------

def invroot_lu(rowptr, colind, vals, rows=None):
    """The submatrix method for p = 1 computed as in the paper's prototype (Sec. 6.1): each
    S_j is inverted through its LU factorisation (LAPACK getrf + getri, which
    ``scipy.linalg.inv`` calls), and Alg. 2 keeps column pos_j of the inverse.  Unlike the
    spectral route it accepts indefinite nonsingular submatrices (raises on a singular
    one).  Same result layout as ``invroot``.  Used as the paper-faithful CPU baseline for
    p = 1; the parity reference stays ``invroot``."""
    import scipy.linalg as sl
    nnz = len(colind)
    out = np.full(nnz, np.nan)
    n = len(rowptr) - 1
    for j in (range(n) if rows is None else rows):
        s, r, pos = submatrix(rowptr, colind, vals, j)
        out[rowptr[j]:rowptr[j + 1]] = sl.inv(s, check_finite=True)[:, pos]
    return out


# ---------------------------------------------------------------------------
# Gradient of a loss on the result with respect to A's stored values
# ---------------------------------------------------------------------------

def divided_differences(lam, p, sign=-1):
    """Gamma_ab = (f(l_a) - f(l_b)) / (l_a - l_b) for f(l) = l^(sign/p), Gamma_aa = f'(l_a).

    With a = l^(1/p):  l_a - l_b = (a_a - a_b) sum_{i<p} a_a^i a_b^(p-1-i).  For
    f(l) = l^(-1/p), f(l_a) - f(l_b) = (a_b - a_a)/(a_a a_b), so the quotient is
    -1 / (a_a a_b sum_i a_a^i a_b^(p-1-i)); for f(l) = l^(1/p) it is
    1 / sum_i a_a^i a_b^(p-1-i).  Neither has cancellation, and on the diagonal they equal
    f'(l) = -(1/p) l^(-1/p-1) and (1/p) l^(1/p-1)."""
    a = lam ** (1.0 / p)
    aa = a[:, None]
    bb = a[None, :]
    ssum = np.zeros((len(a), len(a)))
    for i in range(p):
        ssum += aa ** i * bb ** (p - 1 - i)
    return 1.0 / ssum if sign > 0 else -1.0 / (aa * bb * ssum)


def submatrix_grad(s, pos, g, p, sign=-1):
    """dL/dS for L = <g, column pos of S^(sign/p)>, symmetrised (Daleckii-Krein)."""
    lam, v = np.linalg.eigh(s)
    if lam[0] <= 0.0:
        raise ValueError("submatrix not positive definite")
    m = len(lam)
    gbar = np.zeros((m, m))
    gbar[:, pos] += 0.5 * g
    gbar[pos, :] += 0.5 * g
    gam = divided_differences(lam, p, sign)
    return v @ (gam * (v.T @ gbar @ v)) @ v.T


def grad(rowptr, colind, vals, p, grad_out, sign=-1, rows=None):
    """Gradient of L = sum(grad_out * invroot(A, sign)) with respect to A's stored values.

    For every row j: G_j = dL/dS_j (``submatrix_grad``), then G_j[k][l] is added to the
    stored value at (R_j[k], R_j[l]).  Entries of S_j that are not stored in A are
    constants (zero) and receive nothing.  L is a sum over rows (each row's segment depends
    on S_j alone), so with ``rows`` given the result is the contribution of those rows'
    terms; contributions of disjoint row sets add up to the full gradient."""
    n = len(rowptr) - 1
    out = np.zeros(len(colind))
    for j in (range(n) if rows is None else rows):
        s, r, pos = submatrix(rowptr, colind, vals, j)
        gj = submatrix_grad(s, pos, np.asarray(grad_out[rowptr[j]:rowptr[j + 1]]), p, sign)
        for k in range(len(r)):
            row = r[k]
            cols = np.asarray(colind[rowptr[row]:rowptr[row + 1]], dtype=np.int64)
            where = np.searchsorted(cols, r)
            ok = where < len(cols)
            ok[ok] &= cols[where[ok]] == r[ok]
            np.add.at(out, rowptr[row] + where[ok], gj[k, ok])
    return out


# ---------------------------------------------------------------------------
# Sec. 4.1: residual of an approximate inverse p-th root
# ---------------------------------------------------------------------------

def to_dense(n, rowptr, colind, vals):
    d = np.zeros((n, n))
    for j in range(n):
        d[j, colind[rowptr[j]:rowptr[j + 1]]] = vals[rowptr[j]:rowptr[j + 1]]
    return d


def residual_2norm(a_dense, y_dense, p):
    """||X^p A - I||_2 (Sec. 4.1) for the column-assembled X of Alg. 2.

    The CSR result is row-based (row j holds what Alg. 2 writes into column j), so
    the paper's X is the transpose of the dense CSR result ``y_dense``."""
    x = y_dense.T
    xp = np.linalg.matrix_power(x, p)
    return float(np.linalg.norm(xp @ a_dense - np.eye(a_dense.shape[0]), 2))
