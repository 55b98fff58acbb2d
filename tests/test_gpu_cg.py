"""The preconditioning application (Sec. 4.4) on the GPU: submat_pcg against the CG oracle,
plain and with K ~ A^(-1/2) from the submatrix method (p = 2), on the stand-ins for the
section's SuiteSparse matrices."""
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


def _close_iters(a, b):
    return abs(a - b) <= max(2, int(0.02 * max(a, b)))


@pytest.mark.parametrize("make", [wl.laplace2d_aniso, wl.jump3d])
def test_cg_plain_and_preconditioned(sm, make):
    a = make()
    v = torch.tensor(a.vals, device="cuda")
    b = np.ones(a.n)
    plan = sm.submat_plan(a.rowptr, a.colind, 2, precision="fp64")
    # plain CG: the same iteration count as the oracle, residual at the threshold
    x, it, rel = sm.submat_pcg(plan, v)
    xo, ito, relo, trueo = oracle.cg.solve(a.rowptr, a.colind, a.vals, b)
    assert _close_iters(it, ito) and rel <= 1e-6
    true = np.linalg.norm(b - oracle.cg.spmv(a.rowptr, a.colind, a.vals, x.cpu().numpy()))
    assert true / np.linalg.norm(b) <= 1.5e-6
    # preconditioned with the GPU's K (FP64 path): the oracle CG on the same K agrees
    k = sm.submat_invroot(plan, v)
    xk, itk, relk = sm.submat_pcg(plan, v, vals_k=k)
    kk = k.cpu().numpy()
    xko, itko, relko, trueko = oracle.cg.solve(a.rowptr, a.colind, a.vals, b, vals_k=kk)
    assert _close_iters(itk, itko) and relk <= 1e-6
    assert itk < it                                     # the preconditioner helps
    # the transformed system's residual K^T (b - A x) of the returned x
    res = oracle.cg.spmv_t(a.rowptr, a.colind, kk,
                           b - oracle.cg.spmv(a.rowptr, a.colind, a.vals, xk.cpu().numpy()))
    rhs = oracle.cg.spmv_t(a.rowptr, a.colind, kk, b)
    assert np.linalg.norm(res) / np.linalg.norm(rhs) <= 2e-6


def test_cg_mixed_preconditioner_and_repeatability(sm):
    a = wl.overlap_uniform(n=4096, kappa=1e5)
    v = torch.tensor(a.vals, device="cuda")
    plan = sm.submat_plan(a.rowptr, a.colind, 2)                  # tcgen05 mixed path
    k = sm.submat_invroot(plan, v)
    x1, it1, rel1 = sm.submat_pcg(plan, v, vals_k=k)
    x2, it2, rel2 = sm.submat_pcg(plan, v, vals_k=k)
    torch.cuda.synchronize()
    assert it1 == it2 and torch.equal(x1, x2)              # fixed-order reductions
    _, it0, _ = sm.submat_pcg(plan, v)
    assert rel1 <= 1e-6 and it1 < it0
    _, itko, _, _ = oracle.cg.solve(a.rowptr, a.colind, a.vals, np.ones(a.n),
                                    vals_k=k.cpu().numpy())
    assert _close_iters(it1, itko)


def test_cg_not_positive_definite(sm):
    n = 64
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    plan = sm.submat_plan(rp, ci, 2, precision="fp64")
    v = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_pcg(plan, v)
    assert ei.value.name == "SUBMAT_ENOTSPD"
