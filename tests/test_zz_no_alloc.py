"""The no-allocation entry point (submat_invroot_noalloc) against the FP64 oracle and the
plan-based FP64 path.

Some callers cannot allocate device memory (code inside another framework's memory pool,
allocation-free sections of an application); submat_invroot_noalloc serves them with a
fixed device array inside the library.  This file sorts last so that a run stopping at the
first failure has run every other test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1710_10899_gb300 as pkg
    pkg.load_library()
    return pkg


def row_rel(a, y, ref, rows):
    return np.array([float(np.linalg.norm(y[a.rowptr[j]:a.rowptr[j + 1]] -
                                          ref[a.rowptr[j]:a.rowptr[j + 1]]) /
                           np.linalg.norm(ref[a.rowptr[j]:a.rowptr[j + 1]])) for j in rows])


def dev(a, vals=None, colind=None):
    return (torch.tensor(a.rowptr, device="cuda"),
            torch.tensor(a.colind if colind is None else colind, device="cuda"),
            torch.tensor(a.vals if vals is None else vals, device="cuda"))


@pytest.mark.parametrize("p", [1, 2])
def test_noalloc_matches_plan_path_twice(sm, p):
    for a in (wl.overlap_uniform(n=1500), wl.overlap_small()):
        rp, ci, v = dev(a)
        plan = sm.submat_plan(a.rowptr, a.colind, p, precision="fp64")
        ref = sm.submat_invroot(plan, v, sync=True).cpu().numpy()
        m_max = int(a.row_sizes().max())
        out = torch.full_like(v, float("nan"))
        outs = []
        for _ in range(2):                       # two calls in a row share the array
            sm.submat_invroot_noalloc(rp, ci, p, v, out, m_max=m_max)
            outs.append(out.cpu().numpy().copy())
        for y in outs:
            assert np.isfinite(y).all()
            assert row_rel(a, y, ref, range(a.n)).max() <= 1e-10
        np.testing.assert_array_equal(outs[0], outs[1])


@pytest.mark.parametrize("p", [1, 2, 3])
def test_noalloc_matches_oracle(sm, p):
    a = wl.overlap_small()                       # every row, orders 1..27
    rp, ci, v = dev(a)
    y = sm.submat_invroot_noalloc(rp, ci, p, v).cpu().numpy()
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, p)
    assert row_rel(a, y, ref, range(a.n)).max() <= 1e-10
    b = wl.overlap_uniform(n=1500)               # orders up to ~240, sampled rows
    rp, ci, v = dev(b)
    y = sm.submat_invroot_noalloc(rp, ci, p, v).cpu().numpy()
    rows = list(range(0, b.n, 13)) + [int(np.argmax(b.row_sizes()))]
    ref = oracle.invroot(b.rowptr, b.colind, b.vals, p, rows=rows)
    assert row_rel(b, y, ref, rows).max() <= 1e-10


@pytest.mark.parametrize("p", [1, 2])
def test_noalloc_eigendecomposition_branch(sm, p):
    """Rows whose own diagonal entry is 1e-16 cannot converge in the iteration's 40 steps
    (the smallest eigenvalue of M_0 grows by at most (1 + 1/p)^p per step), so their residual
    test fails and the in-CTA Jacobi eigendecomposition computes them.  The values are
    diagonal inside a dense stored pattern (explicit zeros count), so the exact result is
    a_jj^(-1/p) e_pos, which the oracle's eigendecomposition reproduces."""
    import scipy.linalg as sl
    rng = np.random.default_rng(40 + p)
    d = rng.uniform(1.0, 2.0, 96)
    tiny = [3, 17, 40, 77]
    d[tiny] = 1e-16
    keep = sl.block_diag(*[np.ones((8, 8), bool)] * 12)
    a = wl.dense_to_csr(np.diag(d), keep=keep)
    rp, ci, v = dev(a)
    y = sm.submat_invroot_noalloc(rp, ci, p, v).cpu().numpy()
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, p)
    assert row_rel(a, y, ref, range(a.n)).max() <= 1e-10
    for j in tiny:
        seg = y[a.rowptr[j]:a.rowptr[j + 1]]
        pos = int(np.nonzero(a.colind[a.rowptr[j]:a.rowptr[j + 1]] == j)[0][0])
        assert seg[pos] == pytest.approx(1e-16 ** (-1.0 / p), rel=1e-12)


def test_noalloc_not_spd(sm):
    a = wl.overlap_small(n=500)
    vals = a.vals.copy()
    j = 17
    d = a.rowptr[j] + int(np.nonzero(a.colind[a.rowptr[j]:a.rowptr[j + 1]] == j)[0][0])
    vals[d] = -50.0
    rp, ci, v = dev(a, vals=vals)
    out = torch.zeros_like(v)
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_invroot_noalloc(rp, ci, 2, v, out)
    assert ei.value.name == "SUBMAT_ENOTSPD"
    y = out.cpu().numpy()
    assert np.isnan(y[a.rowptr[j]:a.rowptr[j + 1]]).all()
    affected = {r for r in range(a.n) if j in a.colind[a.rowptr[r]:a.rowptr[r + 1]]}
    good = [r for r in range(a.n) if r not in affected]
    ref = oracle.invroot(a.rowptr, a.colind, vals, 2, rows=good)
    assert row_rel(a, y, ref, good).max() <= 1e-10


def test_noalloc_missing_diagonal(sm):
    n = 50
    off = np.full(n - 1, 0.3)
    dense = 2.0 * np.eye(n) + np.diag(off, 1) + np.diag(off, -1)
    keep = dense != 0
    keep[10, 10] = False
    a = wl.dense_to_csr(dense, keep=keep)
    rp, ci, v = dev(a)
    out = torch.zeros_like(v)
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_invroot_noalloc(rp, ci, 2, v, out)
    assert ei.value.name == "SUBMAT_ENODIAG"
    y = out.cpu().numpy()
    assert np.isnan(y[a.rowptr[10]:a.rowptr[11]]).all()
    good = [r for r in range(n) if abs(r - 10) > 1]
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, 2, rows=good)
    assert row_rel(a, y, ref, good).max() <= 1e-10


def test_noalloc_rejects_out_of_range_column_index(sm):
    """A column index equal to n (one past the last row) is caught by the kernel's checks
    before any address is formed from it: that row is NaN and the call SUBMAT_EINVAL."""
    a = wl.overlap_small(n=200)
    ci = a.colind.copy()
    j = 3
    ci[a.rowptr[j + 1] - 1] = a.n                # the row's last (largest) index
    rp, cit, v = dev(a, colind=ci)
    out = torch.zeros_like(v)
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_invroot_noalloc(rp, cit, 2, v, out, m_max=int(a.row_sizes().max()))
    assert ei.value.name == "SUBMAT_EINVAL"
    y = out.cpu().numpy()
    assert np.isnan(y[a.rowptr[j]:a.rowptr[j + 1]]).all()


def test_noalloc_rejects_rows_longer_than_m_max(sm):
    a = wl.overlap_small(n=300)
    rp, ci, v = dev(a)
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_invroot_noalloc(rp, ci, 2, v, torch.empty_like(v), m_max=2)
    assert ei.value.name == "SUBMAT_ETOOBIG"
