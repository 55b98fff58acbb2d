"""FP64 CPU oracle of the preconditioning application (Lass et al., PASC'18, Sec. 4.4,
"Preconditioning"): the conjugate gradient method on A x = b, plain and with the
submatrix method's K ~ A^(-1/2) applied as K^T A K y = K^T b, x = K y.

TEST INFRASTRUCTURE ONLY (see ``oracle/submatrix.py``): imported by ``tests/`` and
nothing on the product path.  Plain numpy; the sparse products are written out from the
CSR arrays (a weighted count per row or column).

What it computes, in the section's order:

* b = [1, ..., 1]^T; CG (Hestenes-Stiefel) on the system, stopping when the residual of
  the iterated system falls to ``tol`` times its right-hand side in the 2-norm (the
  section's threshold 1e-6), with at most 2n iterations.
* With K: the operator y -> K^T (A (K y)) and right-hand side K^T b; the returned x is K y.

Readings where the section is silent (also in the design notes):

* "the residual" is that of the system CG iterates on (K^T A K y = K^T b when
  preconditioned), relative to its right-hand side; the true residual ||b - A x|| / ||b||
  is reported beside it.
* K is the CSR result of the submatrix method for p = 2 on A's pattern (the paper's
  storage: row j holds column pos_j of F_j, i.e. K's row j is F_j's column); K is used as
  that CSR matrix, K^T as its transpose.
"""
from __future__ import annotations

import numpy as np


def _rows(rowptr):
    """Row index of every stored entry."""
    return np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))


def spmv(rowptr, colind, vals, x):
    """y = M x for the CSR matrix M: y_i = sum over row i's entries of M_ij x_j."""
    n = len(rowptr) - 1
    return np.bincount(_rows(rowptr), weights=vals * x[colind], minlength=n)


def spmv_t(rowptr, colind, vals, x):
    """y = M^T x for the CSR matrix M: each stored M_ij adds M_ij x_i to y_j."""
    n = len(rowptr) - 1
    return np.bincount(colind, weights=vals * x[_rows(rowptr)], minlength=n)


def cg(apply, b, tol=1e-6, max_iter=None):
    """Conjugate gradients for the SPD operator ``apply``: returns (x, iterations,
    relative residual ||r|| / ||b|| of the recursively updated residual)."""
    n = b.shape[0]
    if max_iter is None:
        max_iter = 2 * n
    x = np.zeros(n)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    bnorm = float(np.sqrt(b @ b))
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    while np.sqrt(rr) > tol * bnorm and it < max_iter:
        ap = apply(p)
        alpha = rr / float(p @ ap)
        x = x + alpha * p
        r = r - alpha * ap
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, float(np.sqrt(rr)) / bnorm


def solve(rowptr, colind, vals_a, b, vals_k=None, tol=1e-6, max_iter=None):
    """A x = b by CG, or by CG on K^T A K y = K^T b with x = K y when vals_k is given (K on
    A's pattern).  Returns (x, iterations, relative residual of the iterated system,
    true relative residual ||b - A x|| / ||b||)."""
    if vals_k is None:
        x, it, rel = cg(lambda v: spmv(rowptr, colind, vals_a, v), b, tol, max_iter)
    else:
        op = lambda v: spmv_t(rowptr, colind, vals_k,
                              spmv(rowptr, colind, vals_a, spmv(rowptr, colind, vals_k, v)))
        y, it, rel = cg(op, spmv_t(rowptr, colind, vals_k, b), tol, max_iter)
        x = spmv(rowptr, colind, vals_k, y)
    true = float(np.linalg.norm(b - spmv(rowptr, colind, vals_a, x)) / np.linalg.norm(b))
    return x, it, rel, true
