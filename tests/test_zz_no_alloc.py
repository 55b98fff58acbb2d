"""The no-allocation entry point (submat_invroot_noalloc) against the plan-based FP64 path.

Some callers cannot allocate device memory (code inside another framework's memory pool,
allocation-free sections of an application); submat_invroot_noalloc serves them with a
fixed device array inside the library.  This file sorts last so that a run stopping at the
first failure has run every other test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

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


def row_max_rel(a, y, ref):
    worst = 0.0
    for j in range(a.n):
        s = slice(a.rowptr[j], a.rowptr[j + 1])
        worst = max(worst, float(np.linalg.norm(y[s] - ref[s]) / np.linalg.norm(ref[s])))
    return worst


@pytest.mark.parametrize("p", [1, 2])
def test_noalloc_matches_plan_path_twice(sm, p):
    for a in (wl.overlap_uniform(n=1500), wl.overlap_small()):
        rp = torch.tensor(a.rowptr, device="cuda")
        ci = torch.tensor(a.colind, device="cuda")
        v = torch.tensor(a.vals, device="cuda")
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
            assert row_max_rel(a, y, ref) <= 1e-10
        np.testing.assert_array_equal(outs[0], outs[1])


def test_noalloc_rejects_rows_longer_than_m_max(sm):
    a = wl.overlap_small(n=300)
    rp = torch.tensor(a.rowptr, device="cuda")
    ci = torch.tensor(a.colind, device="cuda")
    v = torch.tensor(a.vals, device="cuda")
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_invroot_noalloc(rp, ci, 2, v, torch.empty_like(v), m_max=2)
    assert ei.value.name == "SUBMAT_ETOOBIG"
