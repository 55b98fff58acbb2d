"""The seeded input generators (workloads.py) at small sizes: valid CSR for the plan (sorted,
unique, in range, diagonal stored, symmetric pattern and values), every submatrix SPD (the
method needs nothing more), the condition number the diagonal shift aims at, and
repeatable output for a fixed seed."""
import numpy as np
import pytest

import workloads as wl

CASES = {
    "overlap_small": lambda: wl.overlap_small(n=300),
    "overlap_uniform": lambda: wl.overlap_uniform(n=600, kappa=1e3),
    "overlap_grad": lambda: wl.overlap_grad(n=500),
    "overlap_clustered": lambda: wl.overlap_clustered(n=1500),
    "block_overlap": lambda: wl.block_overlap(atoms=40),
    "laplace2d_aniso": lambda: wl.laplace2d_aniso(nx=12),
    "jump3d": lambda: wl.jump3d(nx=6),
    "random_sparse_spd": lambda: wl.random_sparse_spd(40, 0.2, seed=3),
}


def _dense(a):
    return a.to_scipy().toarray()


@pytest.mark.parametrize("name", sorted(CASES))
def test_valid_symmetric_csr_with_spd_submatrices(name):
    a = CASES[name]()
    rp, ci = a.rowptr, a.colind
    assert rp.dtype == np.int32 and ci.dtype == np.int32 and a.vals.dtype == np.float64
    assert rp[0] == 0 and rp[-1] == len(ci) == len(a.vals) and np.all(np.diff(rp) >= 1)
    assert ci.min() >= 0 and ci.max() < a.n
    for j in range(a.n):
        row = ci[rp[j]:rp[j + 1]]
        assert np.all(np.diff(row) > 0)
        assert j in row
    d = _dense(a)
    pattern = np.zeros((a.n, a.n), dtype=bool)
    for j in range(a.n):
        pattern[j, ci[rp[j]:rp[j + 1]]] = True
    assert np.array_equal(pattern, pattern.T)
    assert np.array_equal(d, d.T)
    rng = np.random.default_rng(0)
    for j in rng.choice(a.n, size=min(a.n, 25), replace=False):
        r = ci[rp[j]:rp[j + 1]]
        assert np.linalg.eigvalsh(d[np.ix_(r, r)])[0] > 0.0


@pytest.mark.parametrize("kappa", [1e2, 1e3])
def test_diagonal_shift_sets_the_condition_number(kappa):
    a = wl.overlap_uniform(n=700, kappa=kappa)
    lam = np.linalg.eigvalsh(_dense(a))
    assert lam[0] > 0.0
    assert abs(lam[-1] / lam[0] - kappa) <= 1e-4 * kappa


@pytest.mark.parametrize("name", sorted(CASES))
def test_seeded_generators_repeat(name):
    a, b = CASES[name](), CASES[name]()
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.colind, b.colind)
    assert np.array_equal(a.vals, b.vals)
