"""FP64 CPU oracle of the global refinement of the submatrix result (Lass et al., PASC'18,
Sec. 4.5): the submatrix method's Y ~ A^(-1/p) serves as the initial guess of a Newton
iteration for the inverse p-th root (Bini et al., cited in Sec. 2 and 4.5), with every
product truncated to A's sparsity pattern, as a sparse-times-sparse iteration has to be.

TEST INFRASTRUCTURE ONLY (see ``oracle/submatrix.py``): imported by ``tests/`` and nothing
on the product path.  Dense numpy products restricted to the pattern, for small n.

Readings where the section is silent (also in the design notes):

* The iteration is Newton's for A^(-1/p) from a symmetric guess X:
  R = A X, then R <- R X (p - 1 more times), so R ~ A X^p; X <- ((p + 1) X - X R) / p;
  X <- (X + X^T) / 2.  Every product is truncated to A's pattern (entries outside it are
  dropped), the step's result is symmetrised (the exact iterates are symmetric).
* The start is the symmetric part of the submatrix result, (Y + Y^T) / 2 (Y itself is not
  symmetric, Sec. 3.4).
* With a dense pattern nothing is truncated and the iteration is Newton's, converging
  quadratically to A^(-1/p) from a close start.
"""
from __future__ import annotations

import numpy as np

from .submatrix import to_dense


def _mask(n, rowptr, colind):
    m = np.zeros((n, n), dtype=bool)
    for i in range(n):
        m[i, colind[rowptr[i]:rowptr[i + 1]]] = True
    return m


def _vals(d, rowptr, colind):
    n = len(rowptr) - 1
    return np.concatenate([d[i, colind[rowptr[i]:rowptr[i + 1]]] for i in range(n)])


def masked_product(rowptr, colind, lv, rv):
    """(L R) restricted to the pattern, L and R given by their values on the pattern."""
    n = len(rowptr) - 1
    lo = to_dense(n, rowptr, colind, lv)
    ro = to_dense(n, rowptr, colind, rv)
    return _vals(lo @ ro, rowptr, colind)


def symmetrize(rowptr, colind, v):
    n = len(rowptr) - 1
    d = to_dense(n, rowptr, colind, v)
    return _vals(0.5 * (d + d.T), rowptr, colind)


def refine(rowptr, colind, a_vals, y_vals, p, iters):
    """``iters`` truncated Newton steps from the symmetric part of y; returns the values of
    every iterate (the start first)."""
    x = symmetrize(rowptr, colind, y_vals)
    out = [x]
    for _ in range(iters):
        r = masked_product(rowptr, colind, a_vals, x)
        for _ in range(p - 1):
            r = masked_product(rowptr, colind, r, x)
        x = ((p + 1) * x - masked_product(rowptr, colind, x, r)) / p
        x = symmetrize(rowptr, colind, x)
        out.append(x)
    return out


def error_on_pattern(rowptr, colind, a_vals, x_vals, p):
    """||X - (A^(-1/p) restricted to the pattern)||_F / ||A^(-1/p) restricted||_F, with
    A^(-1/p) from the dense symmetric eigendecomposition."""
    n = len(rowptr) - 1
    a = to_dense(n, rowptr, colind, a_vals)
    lam, v = np.linalg.eigh(a)
    z = (v * lam ** (-1.0 / p)) @ v.T
    zp = _vals(z, rowptr, colind)
    return float(np.linalg.norm(x_vals - zp) / np.linalg.norm(zp))
