"""The autograd wrapper's host logic with a stand-in plan (no GPU): the backward goes
through the plan's backward, and a backward through an earlier forward of the same plan,
whose saved input the plan no longer holds, raises instead of returning a gradient at the
wrong point."""
import pytest

torch = pytest.importorskip("torch")


class _Plan:
    """Duck-typed stand-in for paper_1710_10899_gb300.Plan: y = 2 v, dL/dv = 2 g."""

    def __init__(self):
        self._fwd_gen = 0

    def invroot(self, v):
        self._fwd_gen += 1
        return 2.0 * v.detach()

    def backward(self, g):
        return 2.0 * g


def test_backward_goes_through_the_plan():
    import paper_1710_10899_gb300 as sm
    v = torch.ones(5, dtype=torch.float64, requires_grad=True)
    y = sm.SubmatInvRoot.apply(v, _Plan())
    (3.0 * y).sum().backward()
    assert torch.equal(v.grad, torch.full((5,), 6.0, dtype=torch.float64))


def test_backward_through_a_stale_forward_raises():
    import paper_1710_10899_gb300 as sm
    plan = _Plan()
    v = torch.ones(5, dtype=torch.float64, requires_grad=True)
    y1 = sm.SubmatInvRoot.apply(v, plan)
    y2 = sm.SubmatInvRoot.apply(v, plan)
    y2.sum().backward()                       # the latest forward: fine
    with pytest.raises(RuntimeError, match="another forward"):
        y1.sum().backward()
