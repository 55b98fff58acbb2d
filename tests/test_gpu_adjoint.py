"""The Daleckii-Krein adjoint on the GPU against the FP64 oracle gradient and against
central finite differences of the GPU forward (FP64 path)."""
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


@pytest.mark.parametrize("p", [1, 2, 3])
def test_grad_matches_oracle(sm, p):
    a = wl.overlap_uniform(n=500, kappa=1e3)
    w = wl.random_on_pattern(a, seed=1)
    plan = sm.submat_plan(a.rowptr, a.colind, p)
    v = torch.tensor(a.vals, device="cuda")
    sm.submat_invroot(plan, v)
    g = sm.submat_invroot_backward(plan, torch.tensor(w, device="cuda")).cpu().numpy()
    gref = oracle.grad(a.rowptr, a.colind, a.vals, p, w)
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) <= 1e-10
    assert np.abs(g - gref).max() <= 1e-10 * np.abs(gref).max()


def test_grad_shared_memory_layouts(sm):
    """Rows whose Jacobi keeps the eigenvectors next to the packed triangle in shared memory
    (order 100), only the triangle (order 200), or works in global memory (order 260), on
    one block-diagonal pattern, against the oracle gradient."""
    import scipy.linalg as sl
    rng = np.random.default_rng(17)
    sizes = [100, 200, 260]
    blocks = []
    for n in sizes:
        q = rng.standard_normal((n, n))
        blocks.append(q @ q.T / n + 0.5 * np.eye(n))
    a = wl.dense_to_csr(sl.block_diag(*blocks),
                        keep=sl.block_diag(*[np.ones((n, n), dtype=bool) for n in sizes]))
    w = wl.random_on_pattern(a, seed=4)
    plan = sm.submat_plan(a.rowptr, a.colind, 2)
    sm.submat_invroot(plan, torch.tensor(a.vals, device="cuda"))
    g = sm.submat_invroot_backward(plan, torch.tensor(w, device="cuda")).cpu().numpy()
    gref = oracle.grad(a.rowptr, a.colind, a.vals, 2, w)
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) <= 1e-10
    assert np.abs(g - gref).max() <= 1e-10 * np.abs(gref).max()


@pytest.mark.parametrize("p", [2, 3])
def test_positive_root_grad_matches_oracle(sm, p):
    a = wl.overlap_uniform(n=400, kappa=1e3)
    w = wl.random_on_pattern(a, seed=2)
    plan = sm.submat_plan(a.rowptr, a.colind, p, root_sign=1)
    v = torch.tensor(a.vals, device="cuda")
    sm.submat_invroot(plan, v)
    g = sm.submat_invroot_backward(plan, torch.tensor(w, device="cuda")).cpu().numpy()
    gref = oracle.grad(a.rowptr, a.colind, a.vals, p, w, sign=1)
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) <= 1e-10


def test_autograd_and_central_differences(sm):
    a = wl.overlap_grad(n=2048)                 # the differentiation workload, scaled down
    w = torch.tensor(wl.random_on_pattern(a, seed=1), device="cuda")
    plan = sm.submat_plan(a.rowptr, a.colind, 2, precision="fp64")
    vals = torch.tensor(a.vals, device="cuda", requires_grad=True)
    y = sm.SubmatInvRoot.apply(vals, plan)
    (w * y).sum().backward()
    grad = vals.grad.detach().clone()
    fplan = sm.submat_plan(a.rowptr, a.colind, 2, precision="fp64")

    def loss(x):
        return float((w * sm.submat_invroot(fplan, x)).sum())

    h = 1e-6
    base = torch.tensor(a.vals, device="cuda")
    for seed in range(4):
        e = torch.tensor(wl.random_on_pattern(a, seed=100 + seed, symmetric=True), device="cuda")
        e /= e.norm()
        fd = (loss(base + h * e) - loss(base - h * e)) / (2 * h)
        ad = float((grad * e).sum())
        assert abs(fd - ad) <= 1e-6 * max(1.0, abs(fd)), (seed, fd, ad)


@pytest.mark.parametrize("wave_mib", [0, 1])
def test_deterministic_grad(sm, wave_mib):
    """The atomic-free backward (fixed summation order per stored entry, in one wave or in
    many 1 MiB waves) gives identical bits on every call and agrees with the atomic scatter
    and with the oracle gradient."""
    a = wl.overlap_uniform(n=600, kappa=1e3)
    w = torch.tensor(wl.random_on_pattern(a, seed=4), device="cuda")
    v = torch.tensor(a.vals, device="cuda")
    det = sm.submat_plan(a.rowptr, a.colind, 2, grad_deterministic=True, grad_wave_mib=wave_mib)
    sm.submat_invroot(det, v)
    g1 = sm.submat_invroot_backward(det, w)
    g2 = sm.submat_invroot_backward(det, w)
    g3 = sm.submat_invroot_backward(det, w)
    torch.cuda.synchronize()
    assert torch.equal(g1, g2) and torch.equal(g1, g3)
    ato = sm.submat_plan(a.rowptr, a.colind, 2)
    sm.submat_invroot(ato, v)
    ga = sm.submat_invroot_backward(ato, w)
    g = g1.cpu().numpy()
    assert np.abs(g - ga.cpu().numpy()).max() <= 1e-12 * np.abs(g).max()
    gref = oracle.grad(a.rowptr, a.colind, a.vals, 2, w.cpu().numpy())
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) <= 1e-10
