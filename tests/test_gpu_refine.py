"""The global refinement of Sec. 4.5 on the GPU (submat_refine) against its FP64 oracle
(oracle/refine.py): Newton's step for A^(-1/p) with every product restricted to a pattern."""
import numpy as np
import pytest
import scipy.sparse as sp

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


def square_pattern(a):
    """A^2's pattern (it holds A's), with A's values on it (zero where A stores nothing)."""
    m = a.to_scipy()
    pat = (abs(m) @ abs(m)).tocsr()
    pat.sort_indices()
    dense = m.toarray()
    rows = np.repeat(np.arange(a.n), np.diff(pat.indptr))
    vals = dense[rows, pat.indices].astype(np.float64)
    return wl.CSR(a.n, pat.indptr.astype(np.int32), pat.indices.astype(np.int32),
                  np.ascontiguousarray(vals), a.name + "^2")


@pytest.mark.parametrize("p", [1, 2])
def test_refine_matches_oracle_on_a_pattern(sm, p):
    a = wl.overlap_uniform(n=300, kappa=1e3)
    y = oracle.invroot(a.rowptr, a.colind, a.vals, p)
    plan = sm.submat_plan(a.rowptr, a.colind, p, precision="fp64")
    x = sm.submat_refine(plan, torch.tensor(a.vals, device="cuda"), torch.tensor(y, device="cuda"),
                         p, 3).cpu().numpy()
    ref = oracle.refine.refine(a.rowptr, a.colind, a.vals, y, p, 3)[-1]
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-12


def test_refine_p1_on_square_pattern_reduces_the_error(sm):
    """The case where the refinement works (p = 1, Newton-Schulz): the submatrix result on
    A's pattern, extended by zeros to A^2's pattern, refined there.  The GPU iterates equal
    the oracle's and the error against A^(-1) on that pattern falls (from ~0.13 to ~0.02 on
    the block-coefficient operator)."""
    a = wl.jump3d(nx=6)
    a2 = square_pattern(a)
    y = oracle.invroot(a.rowptr, a.colind, a.vals, 1)
    yd = oracle.to_dense(a.n, a.rowptr, a.colind, y)
    rows = np.repeat(np.arange(a2.n), np.diff(a2.rowptr))
    y2 = np.ascontiguousarray(yd[rows, a2.colind])
    plan = sm.submat_plan(a2.rowptr, a2.colind, 1, precision="fp64")
    av = torch.tensor(a2.vals, device="cuda")
    xs = oracle.refine.refine(a2.rowptr, a2.colind, a2.vals, y2, 1, 3)
    errs = []
    for k in range(4):
        x = sm.submat_refine(plan, av, torch.tensor(y2, device="cuda"), 1, k).cpu().numpy()
        assert np.linalg.norm(x - xs[k]) / np.linalg.norm(xs[k]) <= 1e-12
        errs.append(oracle.refine.error_on_pattern(a2.rowptr, a2.colind, a2.vals, x, 1))
    assert errs[-1] < 0.3 * errs[0], errs


@pytest.mark.parametrize("p", [1, 2, 3])
def test_refine_dense_pattern_converges_quadratically(sm, p):
    rng = np.random.default_rng(p)
    b = rng.standard_normal((40, 40))
    dense = b @ b.T / 40 + 0.5 * np.eye(40)
    a = wl.dense_to_csr(dense, keep=np.ones((40, 40), dtype=bool))
    lam = np.linalg.eigvalsh(dense)
    start = oracle.to_dense(a.n, a.rowptr, a.colind, a.vals) * 0.0 + np.eye(40) / lam.max() ** (1.0 / p)
    x0 = np.concatenate([start[i, a.colind[a.rowptr[i]:a.rowptr[i + 1]]] for i in range(a.n)])
    plan = sm.submat_plan(a.rowptr, a.colind, p, precision="fp64")
    av = torch.tensor(a.vals, device="cuda")
    errs = [oracle.refine.error_on_pattern(a.rowptr, a.colind, a.vals,
                                           sm.submat_refine(plan, av, torch.tensor(x0, device="cuda"),
                                                            p, k).cpu().numpy(), p)
            for k in (0, 10, 14)]
    assert errs[-1] <= 1e-12 and errs[1] < errs[0]


def test_refine_repeatable_and_in_place(sm):
    a = wl.overlap_uniform(n=300, kappa=1e3)
    y = torch.tensor(oracle.invroot(a.rowptr, a.colind, a.vals, 1), device="cuda")
    plan = sm.submat_plan(a.rowptr, a.colind, 1, precision="fp64")
    av = torch.tensor(a.vals, device="cuda")
    x1 = sm.submat_refine(plan, av, y, 1, 2)
    x2 = sm.submat_refine(plan, av, y, 1, 2)
    assert torch.equal(x1, x2)
    z = y.clone()
    sm.submat_refine(plan, av, z, 1, 2, x_out=z)
    assert torch.equal(z, x1)
