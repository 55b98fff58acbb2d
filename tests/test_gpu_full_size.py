"""Parity at the workloads' stated sizes.

* uneven batching, n = 131072 (row sizes 7..1113) and the block-sparse Gaussian-basis
  workload at 20000 atoms (n = 260000, sizes 546..1274): mixed path, p = 2, a seeded sample
  of 4096 rows stratified by size (seed 3; the smallest and largest rows included) against
  the FP64 oracle at 1e-6;
* the differentiation workload, n = 16384: the adjoint against the oracle's gradient over
  every stored entry (1e-10) and against central differences (step 1e-6, FP64 forward) on
  32 random sparse symmetric directions of unit norm (seeds 2000..2031), each error at most
  1e-6 of the directions' RMS derivative.

The oracle runs in spawned worker processes on the host cores (this process has already
made CUDA calls, so it must not fork).
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


def row_errors(a, y, ref, rows):
    return np.array([float(np.linalg.norm(y[a.rowptr[j]:a.rowptr[j + 1]] -
                                          ref[a.rowptr[j]:a.rowptr[j + 1]]) /
                           np.linalg.norm(ref[a.rowptr[j]:a.rowptr[j + 1]])) for j in rows])


def forward(sm, a, p, precision):
    plan = sm.submat_plan(a.rowptr, a.colind, p, precision=precision)
    v = torch.tensor(a.vals, device="cuda")
    y = sm.submat_invroot(plan, v, sync=True).cpu().numpy()
    rep = plan.report()
    del plan, v
    torch.cuda.empty_cache()
    return y, rep


@pytest.mark.parametrize("name", ["overlap_clustered", "block_overlap"])
def test_stated_size_stratified_sample(sm, name):
    a = wl.WORKLOADS[name]()
    m = a.row_sizes()
    rows = wl.stratified_rows(m, 4096, seed=3)
    assert m[rows].max() == m.max() and m[rows].min() == m.min()
    if name == "overlap_clustered":
        assert a.n == 131072 and m.max() > 1024
    else:
        assert a.n == 260000 and m.max() > 1200
    y, rep = forward(sm, a, 2, "mixed")
    assert rep["n_notspd"] == 0 and rep["n_rows"] == a.n
    assert np.isfinite(y).all()
    ref = oracle.pool.invroot(a.rowptr, a.colind, a.vals, 2, rows=rows)
    err = row_errors(a, y, ref, rows)
    assert err.max() <= 1e-6, (err.max(), int(rows[int(np.argmax(err))]))


def test_adjoint_stated_size(sm):
    a = wl.overlap_grad()                        # n = 16384, ~130 entries per row
    assert a.n == 16384
    w_np = wl.random_on_pattern(a, seed=1)
    w = torch.tensor(w_np, device="cuda")
    plan = sm.submat_plan(a.rowptr, a.colind, 2, precision="fp64")
    base = torch.tensor(a.vals, device="cuda")
    sm.submat_invroot(plan, base)
    g = sm.submat_invroot_backward(plan, w)
    torch.cuda.synchronize()
    gh = g.cpu().numpy()
    gref = oracle.pool.grad(a.rowptr, a.colind, a.vals, 2, w_np)
    assert np.linalg.norm(gh - gref) / np.linalg.norm(gref) <= 1e-10
    assert np.abs(gh - gref).max() <= 1e-10 * np.abs(gref).max()

    def loss(x):
        y = sm.submat_invroot(plan, x)
        return float(torch.dot(w, y))

    h = 1e-6
    fd, ad = [], []
    for k in range(32):
        e = torch.tensor(wl.random_on_pattern(a, seed=2000 + k, symmetric=True), device="cuda")
        e /= e.norm()
        fd.append((loss(base + h * e) - loss(base - h * e)) / (2 * h))
        ad.append(float(torch.dot(g, e)))
    fd, ad = np.array(fd), np.array(ad)
    # The forward's FP64 rounding leaves ~1e-15 relative noise in L, i.e. ~1e-13 absolute,
    # which the step turns into ~1e-7 of a typical directional derivative; a direction
    # whose derivative happens to be small would magnify it.  Each error is therefore
    # measured against the directions' RMS derivative.
    scale = float(np.sqrt(np.mean(ad ** 2)))
    err = np.abs(fd - ad) / scale
    assert err.max() <= 1e-6, (err.max(), err, ad)
