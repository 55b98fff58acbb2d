"""The bounded device waits of the tensor-core forward, exercised without a GPU fault.

submat_test_stall makes every CTA of the next forwards wait first on a pipeline barrier
that nothing signals, before any copy or tensor-core operation is issued.  The wait must
give up by itself, the call must report SUBMAT_ETIMEOUT with every row NaN, and the same
plan must give its normal result once the flag is cleared.
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


@pytest.mark.parametrize("use_graph", [True, False])
def test_wait_timeout_is_reported_and_the_plan_recovers(sm, use_graph):
    a = wl.overlap_uniform(n=1500)
    # every row on the tcgen05 engine (the small engine, which has no pipeline waits, would
    # take the rows of order <= 32 otherwise)
    plan = sm.submat_plan(a.rowptr, a.colind, 2, use_graph=use_graph, small_max_m=0)
    v = torch.tensor(a.vals, device="cuda")
    out = torch.zeros_like(v)
    ref = sm.submat_invroot(plan, v, out, sync=True).clone()
    assert torch.isfinite(ref).all()
    plan.test_stall(True)
    out.zero_()
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_invroot(plan, v, out, sync=True)
    assert ei.value.name == "SUBMAT_ETIMEOUT"
    assert torch.isnan(out).all()
    assert plan.report()["n_rows"] == a.n
    plan.test_stall(False)
    y = sm.submat_invroot(plan, v, out, sync=True)
    assert torch.equal(y, ref)


def test_wait_timeout_leaves_the_other_engines_rows(sm):
    """With the default size buckets the rows of order <= 32 run on the small engine, which
    the flag does not touch: they keep their values, the others are NaN."""
    a = wl.overlap_uniform(n=1500)
    m = a.row_sizes()
    assert (m <= 32).any() and (m > 32).any()
    plan = sm.submat_plan(a.rowptr, a.colind, 2)
    v = torch.tensor(a.vals, device="cuda")
    ref = sm.submat_invroot(plan, v, sync=True).cpu().numpy()
    plan.test_stall(True)
    out = torch.zeros_like(v)
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_invroot(plan, v, out, sync=True)
    assert ei.value.name == "SUBMAT_ETIMEOUT"
    plan.test_stall(False)
    y = out.cpu().numpy()
    for j in range(a.n):
        seg = slice(a.rowptr[j], a.rowptr[j + 1])
        if m[j] <= 32:
            assert np.array_equal(y[seg], ref[seg])
        else:
            assert np.isnan(y[seg]).all()
