"""Pins for the FP64 oracle: facts the paper and the mathematics fix, independent of the
oracle's own eigendecomposition route.

* dense pattern  -> every row is column j of the full A^(-1/p) (Sec. 3: no truncation),
  checked with Schur-Pade ``fractional_matrix_power`` and, for p=1, Cholesky solves;
* block-diagonal -> blockwise A^(-1/p);
* diagonal A     -> a_jj^(-1/p);
* 4-node chain, p=1 -> exact rationals worked by hand from Alg. 1/2;
* 2x2 submatrices -> the closed-form square root of a 2x2 SPD matrix;
* invariants (F^p S = I, F = F^T), scaling, permutation equivariance;
* tiny random cases against a 40-digit mpmath eigen-solver;
* the paper's Alg. 2 column assembly written out with dense loops (layout pin);
* the gradient against central differences and the Frechet block identity
  f([[S,E],[0,S]]) = [[f(S), L_f(S,E)],[0,f(S)]].
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import workloads as wl


def _dense_spd(n, seed, shift=1.0):
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((n, n))
    return b @ b.T / n + shift * np.eye(n)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_dense_pattern_is_full_inverse_root(p):
    a = _dense_spd(24, seed=p)
    csr = wl.dense_to_csr(a, keep=np.ones_like(a, dtype=bool))
    y = oracle.invroot(csr.rowptr, csr.colind, csr.vals, p)
    full = np.real(sl.fractional_matrix_power(a, -1.0 / p))
    ydense = oracle.to_dense(csr.n, csr.rowptr, csr.colind, y)
    np.testing.assert_allclose(ydense, full.T, rtol=0, atol=1e-12)
    if p == 1:
        c = sl.cho_factor(a)
        np.testing.assert_allclose(ydense, sl.cho_solve(c, np.eye(24)).T, atol=1e-12)
    # the paper's residual (Sec. 4.1) vanishes when nothing is truncated
    assert oracle.residual_2norm(a, ydense, p) < 1e-11


@pytest.mark.parametrize("p", [1, 2])
def test_block_diagonal_is_blockwise_root(p):
    sizes = [1, 3, 7, 4]
    blocks = [_dense_spd(s, seed=10 + s) for s in sizes]
    a = sl.block_diag(*blocks)
    keep = sl.block_diag(*[np.ones((s, s), dtype=bool) for s in sizes])
    csr = wl.dense_to_csr(a, keep=keep)
    y = oracle.to_dense(csr.n, csr.rowptr, csr.colind,
                        oracle.invroot(csr.rowptr, csr.colind, csr.vals, p))
    expect = sl.block_diag(*[np.real(sl.fractional_matrix_power(b, -1.0 / p)) for b in blocks])
    np.testing.assert_allclose(y, expect.T, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_diagonal_matrix(p):
    d = np.array([0.5, 2.0, 3.0, 10.0, 1e-3])
    csr = wl.dense_to_csr(np.diag(d))
    y = oracle.invroot(csr.rowptr, csr.colind, csr.vals, p)
    np.testing.assert_allclose(y, d ** (-1.0 / p), rtol=1e-14)


def test_chain4_p1_exact_rationals():
    # A = tridiag(1, 2, 1), n=4.  Hand-worked from Alg. 1 and Alg. 2:
    #  row 0: R={0,1}, S=[[2,1],[1,2]], S^-1=(1/3)[[2,-1],[-1,2]], pos 0 -> (2/3, -1/3)
    #  row 1: R={0,1,2}, S=tridiag(1,2,1) 3x3, det 4,
    #         S^-1=(1/4)[[3,-2,1],[-2,4,-2],[1,-2,3]], pos 1 -> (-1/2, 1, -1/2)
    #  row 2: R={1,2,3}, same S, pos 1                      -> (-1/2, 1, -1/2)
    #  row 3: R={2,3}, 2x2 as row 0, pos 1                  -> (-1/3, 2/3)
    expect = [Fraction(2, 3), Fraction(-1, 3),
              Fraction(-1, 2), Fraction(1), Fraction(-1, 2),
              Fraction(-1, 2), Fraction(1), Fraction(-1, 2),
              Fraction(-1, 3), Fraction(2, 3)]
    a = 2 * np.eye(4) + np.eye(4, k=1) + np.eye(4, k=-1)
    csr = wl.dense_to_csr(a)
    assert csr.rowptr.tolist() == [0, 2, 5, 8, 10]
    y = oracle.invroot(csr.rowptr, csr.colind, csr.vals, 1)
    np.testing.assert_allclose(y, [float(f) for f in expect], atol=1e-15)


def test_paper_lu_route_p1_exact_rationals_and_indefinite():
    """The paper's own p = 1 route (LU inversion per submatrix, Sec. 6.1): the same exact
    rationals as the hand-worked chain above, the full inverse with a dense pattern, and an
    indefinite nonsingular submatrix, which the spectral route rejects and the LU route
    inverts: A = [[1, 2], [2, 1]], det -3, A^-1 = (1/3) [[-1, 2], [2, -1]]."""
    a = 2 * np.eye(4) + np.eye(4, k=1) + np.eye(4, k=-1)
    csr = wl.dense_to_csr(a)
    y = oracle.invroot_lu(csr.rowptr, csr.colind, csr.vals)
    expect = [2 / 3, -1 / 3, -1 / 2, 1, -1 / 2, -1 / 2, 1, -1 / 2, -1 / 3, 2 / 3]
    np.testing.assert_allclose(y, expect, atol=1e-15)
    d = _dense_spd(20, seed=7)
    c = wl.dense_to_csr(d, keep=np.ones_like(d, dtype=bool))
    yd = oracle.to_dense(c.n, c.rowptr, c.colind, oracle.invroot_lu(c.rowptr, c.colind, c.vals))
    np.testing.assert_allclose(yd, sl.cho_solve(sl.cho_factor(d), np.eye(20)).T, atol=1e-12)
    ind = np.array([[1.0, 2.0], [2.0, 1.0]])
    c = wl.dense_to_csr(ind, keep=np.ones((2, 2), dtype=bool))
    np.testing.assert_allclose(oracle.invroot_lu(c.rowptr, c.colind, c.vals),
                               [-1 / 3, 2 / 3, 2 / 3, -1 / 3], atol=1e-15)
    with pytest.raises(ValueError):
        oracle.invroot(c.rowptr, c.colind, c.vals, 1)


def _inv_sqrt_2x2(s):
    # sqrt(S) = (S + sqrt(det) I) / sqrt(tr + 2 sqrt(det)) for 2x2 SPD S
    det = s[0, 0] * s[1, 1] - s[0, 1] * s[1, 0]
    r = (s + np.sqrt(det) * np.eye(2)) / np.sqrt(np.trace(s) + 2 * np.sqrt(det))
    dr = r[0, 0] * r[1, 1] - r[0, 1] * r[1, 0]
    return np.array([[r[1, 1], -r[0, 1]], [-r[1, 0], r[0, 0]]]) / dr


def test_chain_end_rows_2x2_closed_form_p2():
    rng = np.random.default_rng(3)
    n = 9
    off = rng.uniform(-0.9, 0.9, n - 1)
    a = np.diag(rng.uniform(2.0, 3.0, n)) + np.diag(off, 1) + np.diag(off, -1)
    csr = wl.dense_to_csr(a)
    y = oracle.invroot(csr.rowptr, csr.colind, csr.vals, 2)
    f0 = _inv_sqrt_2x2(a[:2, :2])
    np.testing.assert_allclose(y[0:2], f0[:, 0], atol=1e-14)
    fl = _inv_sqrt_2x2(a[-2:, -2:])
    np.testing.assert_allclose(y[-2:], fl[:, 1], atol=1e-14)
    # interior rows: 3x3 submatrix whose corner A[j-1][j+1] is not stored -> zero
    for j in range(1, n - 1):
        s = a[j - 1:j + 2, j - 1:j + 2].copy()
        assert s[0, 2] == 0.0
        f = np.real(sl.fractional_matrix_power(s, -0.5))
        np.testing.assert_allclose(y[csr.rowptr[j]:csr.rowptr[j + 1]], f[:, 1], atol=1e-13)


def test_unstored_entries_are_zero_in_submatrix():
    # A dense matrix whose pattern is banded: entries outside the stored band must be
    # treated as zero even though the dense array holds values there.
    a = _dense_spd(10, seed=5, shift=3.0)
    keep = np.abs(np.subtract.outer(np.arange(10), np.arange(10))) <= 2
    csr = wl.dense_to_csr(a, keep=keep)
    for j in [0, 4, 9]:
        s, r, pos = oracle.submatrix(csr.rowptr, csr.colind, csr.vals, j)
        expect = np.where(keep, a, 0.0)[np.ix_(r, r)]
        np.testing.assert_array_equal(s, expect)
        assert r[pos] == j


@pytest.mark.parametrize("p", [1, 2, 3])
def test_alg2_column_assembly_layout(p):
    # Alg. 2 written out with dense loops: X[R[i]][j] = f(S_j)[i][R.indexof(j)];
    # the row-based CSR result is X transposed (Sec. 3.4).
    a0 = wl.random_sparse_spd(12, 0.3, seed=7)
    a = oracle.to_dense(a0.n, a0.rowptr, a0.colind, a0.vals)
    n = a.shape[0]
    x = np.zeros((n, n))
    for j in range(n):
        r = [i for i in range(n) if a[i][j] != 0]
        s = np.array([[a[r[k]][r[l]] for l in range(len(r))] for k in range(len(r))])
        f = np.real(sl.fractional_matrix_power(s, -1.0 / p))
        for i in range(len(r)):
            x[r[i]][j] = f[i][r.index(j)]
    y = oracle.to_dense(n, a0.rowptr, a0.colind,
                        oracle.invroot(a0.rowptr, a0.colind, a0.vals, p))
    np.testing.assert_allclose(y, x.T, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_submatrix_invariants(p):
    a = wl.overlap_small(n=400)
    for j in range(0, 400, 37):
        s, r, pos = oracle.submatrix(a.rowptr, a.colind, a.vals, j)
        f = oracle.inv_root(s, p)
        np.testing.assert_allclose(f, f.T, atol=1e-13)
        resid = np.linalg.matrix_power(f, p) @ s - np.eye(len(r))
        assert np.abs(resid).max() < 1e-12 * np.linalg.cond(s)
        np.testing.assert_allclose(oracle.inv_root_column(s, pos, p), f[:, pos], atol=1e-14)
        assert np.linalg.eigvalsh(f).min() > 0


@pytest.mark.parametrize("p", [1, 2, 3])
def test_scaling(p):
    a = wl.overlap_small(n=300)
    y1 = oracle.invroot(a.rowptr, a.colind, a.vals, p)
    y2 = oracle.invroot(a.rowptr, a.colind, 7.5 * a.vals, p)
    np.testing.assert_allclose(y2, 7.5 ** (-1.0 / p) * y1, rtol=1e-12,
                               atol=1e-13 * np.abs(y1).max())


def test_permutation_equivariance():
    a0 = wl.random_sparse_spd(15, 0.25, seed=11)
    a = oracle.to_dense(a0.n, a0.rowptr, a0.colind, a0.vals)
    perm = np.random.default_rng(2).permutation(15)
    b = a[np.ix_(perm, perm)]
    cb = wl.dense_to_csr(b)
    ya = oracle.to_dense(15, a0.rowptr, a0.colind, oracle.invroot(a0.rowptr, a0.colind, a0.vals, 2))
    yb = oracle.to_dense(15, cb.rowptr, cb.colind, oracle.invroot(cb.rowptr, cb.colind, cb.vals, 2))
    np.testing.assert_allclose(yb, ya[np.ix_(perm, perm)], atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_bruteforce_mpmath(p):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for seed in range(3):
        a0 = wl.random_sparse_spd(7, 0.4, seed=seed)
        y = oracle.invroot(a0.rowptr, a0.colind, a0.vals, p)
        for j in range(a0.n):
            s, r, pos = oracle.submatrix(a0.rowptr, a0.colind, a0.vals, j)
            lam, v = mp.eigsy(mp.matrix(s.tolist()))
            m = len(r)
            col = [sum(v[k, i] * lam[i] ** (mp.mpf(-1) / p) * v[pos, i] for i in range(m))
                   for k in range(m)]
            np.testing.assert_allclose(y[a0.rowptr[j]:a0.rowptr[j + 1]],
                                       [float(c) for c in col], rtol=0, atol=1e-14)


def test_plan_bruteforce():
    for seed in range(4):
        a0 = wl.random_sparse_spd(20, 0.2, seed=seed)
        dense = oracle.to_dense(a0.n, a0.rowptr, a0.colind, np.ones(a0.nnz))
        m, pos = oracle.plan(a0.rowptr, a0.colind)
        for j in range(a0.n):
            r = [i for i in range(a0.n) if dense[j][i] != 0]
            assert m[j] == len(r)
            assert pos[j] == r.index(j)


def test_missing_diagonal_and_indefinite_are_errors():
    a = np.array([[0.0, 1.0], [1.0, 2.0]])
    csr = wl.dense_to_csr(a, keep=(a != 0))
    with pytest.raises(ValueError):
        oracle.plan(csr.rowptr, csr.colind)
    b = np.array([[1.0, 2.0], [2.0, 1.0]])        # eigenvalues 3, -1
    cb = wl.dense_to_csr(b)
    with pytest.raises(ValueError):
        oracle.invroot(cb.rowptr, cb.colind, cb.vals, 2)


def test_divided_differences_match_plain_quotient():
    lam = np.array([0.3, 0.9, 2.5, 7.0])
    for p in (1, 2, 3):
        g = oracle.divided_differences(lam, p)
        f = lam ** (-1.0 / p)
        for a in range(4):
            for b in range(4):
                if a == b:
                    assert np.isclose(g[a, a], -(1.0 / p) * lam[a] ** (-1.0 / p - 1), rtol=1e-14)
                else:
                    assert np.isclose(g[a, b], (f[a] - f[b]) / (lam[a] - lam[b]), rtol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_submatrix_grad_frechet_block_identity(p):
    rng = np.random.default_rng(20 + p)
    m = 7
    s = _dense_spd(m, seed=p, shift=0.7)
    g = rng.standard_normal(m)
    pos = 3
    e = rng.standard_normal((m, m))
    e = e + e.T
    z = np.block([[s, e], [np.zeros((m, m)), s]])
    lf = np.real(sl.fractional_matrix_power(z, -1.0 / p))[:m, m:]   # L_f(S, E)
    lhs = np.sum(oracle.submatrix_grad(s, pos, g, p) * e)
    rhs = g @ lf[:, pos]
    assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(rhs))


@pytest.mark.parametrize("p", [1, 2])
def test_grad_central_differences(p):
    a = wl.overlap_uniform(n=300, kappa=50.0)
    w = wl.random_on_pattern(a, seed=1)
    gr = oracle.grad(a.rowptr, a.colind, a.vals, p, w)

    def loss(v):
        return float(np.dot(w, oracle.invroot(a.rowptr, a.colind, v, p)))

    h = 1e-6
    for seed in range(3):
        e = wl.random_on_pattern(a, seed=100 + seed, symmetric=True)
        e /= np.linalg.norm(e)
        fd = (loss(a.vals + h * e) - loss(a.vals - h * e)) / (2 * h)
        assert abs(fd - gr @ e) <= 1e-6 * max(1.0, abs(fd))
    # symmetric: the (r,c) and (c,r) entries carry the same value
    d = oracle.to_dense(a.n, a.rowptr, a.colind, gr)
    np.testing.assert_allclose(d, d.T, atol=1e-13)


# ---------------------------------------------------------------------------
# Positive p-th roots (Sec. 4.2): the same method with f(S) = S^(1/p)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1, 2, 3])
def test_positive_root_dense_pattern_is_full_root(p):
    a = _dense_spd(24, seed=40 + p)
    csr = wl.dense_to_csr(a, keep=np.ones_like(a, dtype=bool))
    y = oracle.invroot(csr.rowptr, csr.colind, csr.vals, p, sign=1)
    full = np.real(sl.fractional_matrix_power(a, 1.0 / p))
    ydense = oracle.to_dense(csr.n, csr.rowptr, csr.colind, y)
    np.testing.assert_allclose(ydense, full.T, rtol=0, atol=1e-12)


def test_positive_root_p1_returns_the_stored_values():
    a = wl.overlap_small(n=300)
    y = oracle.invroot(a.rowptr, a.colind, a.vals, 1, sign=1)
    np.testing.assert_allclose(y, a.vals, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_positive_root_diagonal_and_2x2(p):
    d = np.array([0.5, 2.0, 3.0, 10.0, 1e-3])
    csr = wl.dense_to_csr(np.diag(d))
    np.testing.assert_allclose(oracle.invroot(csr.rowptr, csr.colind, csr.vals, p, sign=1),
                               d ** (1.0 / p), rtol=1e-14)
    if p == 2:
        # sqrt of a 2x2 SPD matrix: (M + sqrt(det) I) / sqrt(tr + 2 sqrt(det))
        m2 = np.array([[2.0, 0.7], [0.7, 1.5]])
        sd = np.sqrt(np.linalg.det(m2))
        expect = (m2 + sd * np.eye(2)) / np.sqrt(np.trace(m2) + 2.0 * sd)
        csr2 = wl.dense_to_csr(m2)
        y = oracle.to_dense(2, csr2.rowptr, csr2.colind,
                            oracle.invroot(csr2.rowptr, csr2.colind, csr2.vals, 2, sign=1))
        np.testing.assert_allclose(y, expect.T, atol=1e-15)


@pytest.mark.parametrize("p", [2, 3])
def test_positive_root_submatrix_relations(p):
    # on every submatrix: (S^(1/p))^p = S, and column pos of S^(1/p) = S (S^(-1/p))^(p-1) e_pos
    a = wl.random_sparse_spd(40, 0.15, seed=8)
    for j in range(a.n):
        s, r, pos = oracle.submatrix(a.rowptr, a.colind, a.vals, j)
        f = oracle.inv_root(s, p, sign=1)
        np.testing.assert_allclose(np.linalg.matrix_power(f, p), s, atol=1e-12 * np.abs(s).max())
        e = np.zeros(len(r))
        e[pos] = 1.0
        g = np.linalg.matrix_power(np.real(sl.fractional_matrix_power(s, -1.0 / p)), p - 1) @ e
        np.testing.assert_allclose(oracle.inv_root_column(s, pos, p, sign=1), s @ g, atol=1e-12)


@pytest.mark.parametrize("p", [2, 3])
def test_positive_root_grad_frechet_and_central_differences(p):
    rng = np.random.default_rng(30 + p)
    m = 7
    s = _dense_spd(m, seed=p, shift=0.7)
    g = rng.standard_normal(m)
    e = rng.standard_normal((m, m))
    e = e + e.T
    z = np.block([[s, e], [np.zeros((m, m)), s]])
    lf = np.real(sl.fractional_matrix_power(z, 1.0 / p))[:m, m:]
    lhs = np.sum(oracle.submatrix_grad(s, 2, g, p, sign=1) * e)
    assert abs(lhs - g @ lf[:, 2]) < 1e-11 * max(1.0, abs(lhs))
    a = wl.overlap_uniform(n=200, kappa=50.0)
    w = wl.random_on_pattern(a, seed=1)
    gr = oracle.grad(a.rowptr, a.colind, a.vals, p, w, sign=1)

    def loss(v):
        return float(np.dot(w, oracle.invroot(a.rowptr, a.colind, v, p, sign=1)))

    h = 1e-6
    d = wl.random_on_pattern(a, seed=200, symmetric=True)
    d /= np.linalg.norm(d)
    fd = (loss(a.vals + h * d) - loss(a.vals - h * d)) / (2 * h)
    assert abs(fd - gr @ d) <= 1e-6 * max(1.0, abs(fd))


# --- the preconditioning application (Sec. 4.4): CG oracle pins ---------------------------
def _dense_csr(a):
    n = a.shape[0]
    return (np.arange(0, n * n + 1, n, dtype=np.int32), np.tile(np.arange(n, dtype=np.int32), n),
            a.ravel().astype(np.float64))


def test_cg_products_brute_force():
    """spmv / spmv_t against dense products on a random (value-nonsymmetric) sparse matrix."""
    a = wl.random_sparse_spd(40, 0.2, seed=3)
    v = wl.random_on_pattern(a, seed=5)
    dense = oracle.to_dense(a.n, a.rowptr, a.colind, v)
    x = np.random.default_rng(1).standard_normal(a.n)
    np.testing.assert_allclose(oracle.cg.spmv(a.rowptr, a.colind, v, x), dense @ x, atol=1e-12)
    np.testing.assert_allclose(oracle.cg.spmv_t(a.rowptr, a.colind, v, x), dense.T @ x, atol=1e-12)


def test_cg_terminates_after_distinct_eigenvalues():
    """In exact arithmetic CG ends after as many steps as A has distinct eigenvalues (with
    b touching all of them); on a diagonal with three values it takes three."""
    d = np.array([1.0, 2.0, 5.0] * 4)
    n = d.shape[0]
    rp, ci = np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32)
    x, it, rel, true = oracle.cg.solve(rp, ci, d, np.ones(n), tol=1e-12)
    assert it == 3 and rel <= 1e-12
    np.testing.assert_allclose(x, 1.0 / d, rtol=1e-12)


def test_cg_matches_dense_solve():
    rng = np.random.default_rng(7)
    b_ = rng.standard_normal((30, 30))
    a = b_ @ b_.T + 30 * np.eye(30)
    rp, ci, v = _dense_csr(a)
    b = rng.standard_normal(30)
    x, it, rel, true = oracle.cg.solve(rp, ci, v, b, tol=1e-13)
    np.testing.assert_allclose(x, np.linalg.solve(a, b), rtol=1e-10, atol=1e-12)
    assert true <= 1e-12


def test_pcg_with_exact_inverse_square_root_takes_one_step():
    """On a dense pattern the submatrix method is exact (every submatrix is A), so
    K = A^(-1/2), K^T A K = I and CG on the transformed system ends after one step with
    x = K K^T b = A^(-1) b."""
    rng = np.random.default_rng(11)
    b_ = rng.standard_normal((20, 20))
    a = b_ @ b_.T + 5 * np.eye(20)
    rp, ci, v = _dense_csr(a)
    k = oracle.invroot(rp, ci, v, 2)
    b = np.ones(20)
    x, it, rel, true = oracle.cg.solve(rp, ci, v, b, vals_k=k, tol=1e-10)
    assert it == 1 and true <= 1e-10
    np.testing.assert_allclose(x, np.linalg.solve(a, b), rtol=1e-9)


# --- global refinement experiment (Sec. 4.5): oracle pins ----------------------------------
def test_refine_masked_product_brute_force():
    a = wl.random_sparse_spd(30, 0.25, seed=2)
    lv = wl.random_on_pattern(a, seed=3)
    rv = wl.random_on_pattern(a, seed=4)
    d = oracle.to_dense(a.n, a.rowptr, a.colind, lv) @ oracle.to_dense(a.n, a.rowptr, a.colind, rv)
    got = oracle.refine.masked_product(a.rowptr, a.colind, lv, rv)
    for i in range(a.n):
        for e in range(a.rowptr[i], a.rowptr[i + 1]):
            assert abs(got[e] - d[i, a.colind[e]]) <= 1e-12 * max(1.0, abs(d[i, a.colind[e]]))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_refine_newton_dense_fixed_point_and_quadratic_convergence(p):
    """With a dense pattern nothing is truncated: A^(-1/p) is a fixed point, and from a start
    that commutes with A (a multiple of I inside the convergence region) the error falls
    quadratically."""
    rng = np.random.default_rng(p)
    b_ = rng.standard_normal((16, 16))
    a = b_ @ b_.T / 16 + 0.5 * np.eye(16)
    rp, ci, v = _dense_csr(a)
    lam, vec = np.linalg.eigh(a)
    z = ((vec * lam ** (-1.0 / p)) @ vec.T).ravel()
    xs = oracle.refine.refine(rp, ci, v, z, p, 1)
    np.testing.assert_allclose(xs[1], z, rtol=1e-10, atol=1e-12)
    start = (np.eye(16) / lam.max() ** (1.0 / p)).ravel()
    xs = oracle.refine.refine(rp, ci, v, start, p, 12)
    errs = [oracle.refine.error_on_pattern(rp, ci, v, x, p) for x in xs]
    assert errs[-1] <= 1e-12
    k = next(i for i, e in enumerate(errs) if e < 1e-3)
    assert errs[k + 1] <= 10 * errs[k] ** 2          # quadratic once close


@pytest.mark.parametrize("p", [2, 3])
def test_refine_newton_first_order_on_noncommuting_error(p):
    """Why the refinement from the submatrix result fails (Sec. 4.5 reading): the step
    X' = ((p+1) X - X (A X^p)) / p, linearised at Z = A^(-1/p) with X = Z + E and E in A's
    eigenbasis, multiplies E_ab by g(z_b / z_a), g(s) = (p - sum_{k<p} s^k) / p (z = the
    eigenvalues of Z); the symmetrisation averages g(s) and g(1/s).  Errors within one
    eigenvalue (s = 1) vanish to first order (quadratic convergence), errors that couple
    eigenvalues far apart are amplified.  A = diag(1, 100), dense pattern (no truncation):
    the off-diagonal error of Z + eps E is multiplied by exactly that average (-2.025 for
    p = 2), the diagonal moves by O(eps^2)."""
    lam = np.array([1.0, 100.0])
    z = lam ** (-1.0 / p)
    rp = np.array([0, 2, 4], dtype=np.int32)
    ci = np.array([0, 1, 0, 1], dtype=np.int32)
    av = np.array([1.0, 0.0, 0.0, 100.0])            # stored zeros keep the pattern dense
    s = z[1] / z[0]

    def g(t):
        return (p - sum(t ** k for k in range(p))) / p

    expect = 0.5 * (g(s) + g(1.0 / s))
    assert abs(expect) > 1.0                          # this error component grows
    for eps in (1e-5, 1e-7):
        x0 = np.array([z[0], eps, eps, z[1]])
        x1 = oracle.refine.refine(rp, ci, av, x0, p, 1)[1]
        assert abs(x1[1] / eps - expect) <= 1e-6 * abs(expect)   # Z's off-diagonal is 0
        assert x1[1] == x1[2]                         # symmetrised
        assert max(abs(x1[0] - z[0]), abs(x1[3] - z[1])) <= 100.0 * eps ** 2


def _random_symmetric(n, density, seed):
    rng = np.random.default_rng(seed)
    mask = np.triu(rng.random((n, n)) < density / 2, 1)
    v = rng.uniform(-1.0, 1.0, (n, n)) * mask
    return v + v.T


def _shift_to_kappa(off, kappa):
    lam = np.linalg.eigvalsh(off)
    return off + (lam[-1] - kappa * lam[0]) / (kappa - 1.0) * np.eye(len(off))


@pytest.mark.parametrize("p", [1, 2])
def test_sec41_residual_trends(p):
    """Sec. 4.1's findings, on seeded random sparse SPD matrices (density 0.05, the
    condition number set by a diagonal shift) instead of MATLAB's sprandsym: the residual
    ||X^p A - I||_2 grows with the condition number on a fixed pattern, and at kappa = 2 it
    stays small as n grows."""
    off = _random_symmetric(200, 0.05, seed=200)
    res = []
    for kappa in (2.0, 10.0, 100.0, 1000.0):
        a = _shift_to_kappa(off, kappa)
        c = wl.dense_to_csr(a)
        y = oracle.to_dense(c.n, c.rowptr, c.colind, oracle.invroot(c.rowptr, c.colind, c.vals, p))
        res.append(oracle.residual_2norm(a, y, p))
    assert all(r0 < r1 for r0, r1 in zip(res, res[1:])), res
    for n in (100, 200, 400):
        a = _shift_to_kappa(_random_symmetric(n, 0.05, seed=n), 2.0)
        c = wl.dense_to_csr(a)
        y = oracle.to_dense(c.n, c.rowptr, c.colind, oracle.invroot(c.rowptr, c.colind, c.vals, p))
        assert oracle.residual_2norm(a, y, p) < 0.15


def test_refine_newton_p1_is_indifferent_to_commutation():
    """For p = 1 the step is Newton-Schulz for the inverse, X' = 2X - X A X: g(s) = 0 for
    every eigenvalue pair, so an error coupling eigenvalues 100 apart vanishes to first
    order (the error after the step is O(eps^2)), unlike p >= 2 above."""
    rp = np.array([0, 2, 4], dtype=np.int32)
    ci = np.array([0, 1, 0, 1], dtype=np.int32)
    av = np.array([1.0, 0.0, 0.0, 100.0])
    z = np.array([1.0, 0.01])
    for eps in (1e-4, 1e-6):
        x0 = np.array([z[0], eps, eps, z[1]])
        x1 = oracle.refine.refine(rp, ci, av, x0, 1, 1)[1]
        err = np.abs(x1 - np.array([z[0], 0.0, 0.0, z[1]])).max()
        assert err <= 200.0 * eps ** 2
