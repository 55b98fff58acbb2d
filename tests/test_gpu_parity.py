"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Error metric: per row j, ||y_j - y_j^oracle||_2 / ||y_j^oracle||_2, maximum over the rows
checked.  Bars: 1e-10 on the FP64 path, 1e-6 on the mixed-precision path; integer plan
bit-exact.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-6}


@pytest.fixture(scope="module")
def sm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1710_10899_gb300 as pkg
    pkg.load_library()
    return pkg


def row_errors(a, y, ref, rows):
    errs = []
    for j in rows:
        s = slice(a.rowptr[j], a.rowptr[j + 1])
        errs.append(np.linalg.norm(y[s] - ref[s]) / np.linalg.norm(ref[s]))
    return np.array(errs)


def run(sm, a, p, precision, **kw):
    plan = sm.submat_plan(a.rowptr, a.colind, p, precision=precision, **kw)
    v = torch.tensor(a.vals, device="cuda", dtype=torch.float64)
    y = sm.submat_invroot(plan, v, sync=True)
    torch.cuda.synchronize()
    return plan, y.cpu().numpy()


def sample_rows(a, k, seed=0):
    m = a.row_sizes()
    rng = np.random.default_rng(seed)
    rows = set(rng.choice(a.n, size=min(k, a.n), replace=False).tolist())
    rows |= {int(np.argmin(m)), int(np.argmax(m))}
    return sorted(rows)


def test_plan_rows_bitexact(sm):
    for a in [wl.overlap_small(), wl.random_sparse_spd(50, 0.2, seed=3),
              wl.overlap_uniform(n=3000)]:
        plan = sm.submat_plan(a.rowptr, a.colind, 2)
        m, pos = plan.rows()
        mo, po = oracle.plan(a.rowptr, a.colind)
        np.testing.assert_array_equal(m, mo)
        np.testing.assert_array_equal(pos, po)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_small_workload_all_rows(sm, precision):
    a = wl.overlap_small()                       # n=2000, m 1..27, p=2
    plan, y = run(sm, a, 2, precision)
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, 2)
    err = row_errors(a, y, ref, range(a.n))
    assert err.max() <= TOL[precision], err.max()
    rep = plan.report()
    assert rep["n_notspd"] == 0


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uniform_sampled(sm, p, precision):
    a = wl.overlap_uniform(n=4096)               # m 31..240: several tiles, ragged tails
    plan, y = run(sm, a, p, precision)
    rows = sample_rows(a, 150, seed=p)
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, p, rows=rows)
    err = row_errors(a, y, ref, rows)
    assert err.max() <= TOL[precision], err.max()
    assert np.isfinite(y).all()


def test_full_size_uniform_sampled(sm):
    a = wl.overlap_uniform()                     # n=32768, m 32..255, kappa 1e3
    plan, y = run(sm, a, 2, "mixed")
    rows = sample_rows(a, 120, seed=5)
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, 2, rows=rows)
    err = row_errors(a, y, ref, rows)
    assert err.max() <= TOL["mixed"], err.max()
    assert np.isfinite(y).all()
    rep = plan.report()
    assert rep["n_notspd"] == 0 and rep["n_rows"] == a.n


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_edge_patterns(sm, precision):
    rng = np.random.default_rng(4)
    cases = []
    d = rng.uniform(0.5, 4.0, 37)
    cases.append(wl.dense_to_csr(np.diag(d)))                                    # m = 1
    off = rng.uniform(-0.9, 0.9, 39)
    cases.append(wl.dense_to_csr(np.diag(rng.uniform(2, 3, 40)) + np.diag(off, 1)
                                 + np.diag(off, -1)))                            # m = 2, 3
    b = rng.standard_normal((70, 70))
    dense = b @ b.T / 70 + np.eye(70)
    cases.append(wl.dense_to_csr(dense, keep=np.ones((70, 70), dtype=bool)))     # one size
    import scipy.linalg as sl
    blocks = []
    for s in [1, 5, 64, 65, 129]:
        q = rng.standard_normal((s, s))
        blocks.append(q @ q.T / s + 0.5 * np.eye(s))
    cases.append(wl.dense_to_csr(sl.block_diag(*blocks),
                                 keep=sl.block_diag(*[np.ones((s, s), bool) for s in
                                                      [1, 5, 64, 65, 129]])))
    for a in cases:
        for p in (1, 2):
            plan, y = run(sm, a, p, precision)
            ref = oracle.invroot(a.rowptr, a.colind, a.vals, p)
            err = row_errors(a, y, ref, range(a.n))
            assert err.max() <= TOL[precision], (a.name, p, err.max())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("p", [1, 2])
def test_algorithmic_flop_count(sm, precision, p):
    """flops_alg counts (p+1) dense products of the true order per executed iteration, plus
    p = 1's final X product: with every row of one order m (dense 40 x 40 blocks) it is
    (p+1) 2 m^3 iters_sum (+ 2 m^3 per row for p = 1)."""
    import scipy.linalg as sl
    rng = np.random.default_rng(31)
    blocks = []
    for _ in range(12):
        q = rng.standard_normal((40, 40))
        blocks.append(q @ q.T / 40 + 0.5 * np.eye(40))
    a = wl.dense_to_csr(sl.block_diag(*blocks),
                        keep=sl.block_diag(*[np.ones((40, 40), bool)] * 12))
    plan, y = run(sm, a, p, precision)
    rep = plan.report()
    m3 = 40.0 ** 3
    expect = (p + 1) * 2 * m3 * rep["iters_sum"] + (2 * m3 * a.n if p == 1 else 0.0)
    assert rep["iters_sum"] > 0
    assert rep["flops_alg"] == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("sign", [-1, 1])
def test_small_engine_all_rows(sm, p, sign):
    """Orders 1..27: every row runs on the small-submatrix engine (working set in shared
    memory, warp-level mma.sync tiles)."""
    a = wl.overlap_small()
    plan, y = run(sm, a, p, "mixed", root_sign=sign, small_max_m=32)
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, p, sign=sign)
    assert row_errors(a, y, ref, range(a.n)).max() <= TOL["mixed"]
    rep = plan.report()
    # a submatrix whose condition estimate exceeds kappa_max goes to the FP64 fallback
    assert rep["n_notspd"] == 0 and rep["n_fallback"] <= 2 and rep["iters_sum"] > a.n


@pytest.mark.parametrize("buckets", [(0, 0), (32, 0), (32, 64), (16, 48), (0, 1536)])
def test_engine_buckets(sm, buckets):
    """Rows routed by order to the small engine, the mma.sync engine and the tcgen05 engine
    (one persistent launch each) all meet the bar, on the uneven workload at 1/8 scale
    (orders 10..596), checked on a sample stratified by size."""
    small, sync = buckets
    a = wl.overlap_clustered(n=16384)
    plan, y = run(sm, a, 2, "mixed", small_max_m=small, sync_max_m=sync)
    rows = wl.stratified_rows(a.row_sizes(), 240, seed=3)
    ref = oracle.pool.invroot(a.rowptr, a.colind, a.vals, 2, rows=rows)
    assert row_errors(a, y, ref, rows).max() <= TOL["mixed"]
    rep = plan.report()
    assert rep["n_fallback"] == 0 and rep["n_rows"] == a.n


@pytest.mark.parametrize("p", [4, 7, 10])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_higher_root_orders(sm, p, precision):
    """Roots beyond the paper's p <= 3, up to the mixed modes' limit SUBMAT_MIXED_MAX_P: the
    exponent bias grows with p (alpha' = alpha 2^(9-b) must stay an FP16 integer), so these
    rows run with fewer bits than p = 2's."""
    assert p <= sm.SUBMAT_MIXED_MAX_P
    a = wl.overlap_uniform(n=2048)
    plan, y = run(sm, a, p, precision)
    rows = sample_rows(a, 100, seed=p)
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, p, rows=rows)
    assert row_errors(a, y, ref, rows).max() <= TOL[precision]
    assert plan.report()["n_notspd"] == 0


def test_dense_pattern_equals_full_root(sm):
    import scipy.linalg as sl
    rng = np.random.default_rng(9)
    b = rng.standard_normal((100, 100))
    dense = b @ b.T / 100 + 0.3 * np.eye(100)
    a = wl.dense_to_csr(dense, keep=np.ones((100, 100), dtype=bool))
    plan, y = run(sm, a, 2, "mixed")
    full = np.real(sl.fractional_matrix_power(dense, -0.5))
    yd = oracle.to_dense(a.n, a.rowptr, a.colind, y)
    assert np.abs(yd - full.T).max() / np.abs(full).max() < 1e-6


def test_clustered_uneven_sizes(sm):
    # the uneven-batching workload at 1/8 scale (orders 10..596): the largest and smallest
    # rows and a random sample against the oracle (orders above 1024: test_order_above_1024)
    a = wl.overlap_clustered(n=16384)
    m = a.row_sizes()
    plan, y = run(sm, a, 2, "mixed")
    order = np.argsort(m)
    rows = sorted(set(order[-4:].tolist()) | set(order[:2].tolist()) | set(sample_rows(a, 20, seed=5)))
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, 2, rows=rows)
    assert m.max() > 4 * m.min()
    assert row_errors(a, y, ref, rows).max() <= TOL["mixed"]


def test_block_overlap_sampled(sm):
    # the block-sparse Gaussian-basis workload at 800 atoms (n = 10400, orders 546..1235,
    # so the largest rows also take the exponent bias of orders above 1024)
    a = wl.block_overlap(atoms=800)
    m = a.row_sizes()
    plan, y = run(sm, a, 2, "mixed")
    order = np.argsort(m)
    rows = sorted(set(order[-3:].tolist()) | {int(order[0])} | set(sample_rows(a, 8, seed=6)))
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, 2, rows=rows)
    assert m.max() > 1024
    assert row_errors(a, y, ref, rows).max() <= TOL["mixed"]
    assert plan.report()["n_fallback"] == 0


@pytest.mark.parametrize("p", [1, 2])
def test_order_above_1024(sm, p):
    # arrow + band: row 0's submatrix is the whole 1200 x 1200 matrix (padded order 1216),
    # where the mixed path's slices give up one bit to keep level-0 sums exact
    n = 1200
    rng = np.random.default_rng(7)
    dense = np.eye(n) * 2.0
    for k in (1, 2):
        off = 0.15 * rng.uniform(0.5, 1.0, n - k)
        dense += np.diag(off, k) + np.diag(off, -k)
    arrow = 0.02 * rng.uniform(0.5, 1.0, n - 1)
    dense[0, 1:] = arrow
    dense[1:, 0] = arrow
    a = wl.dense_to_csr(dense)
    plan, y = run(sm, a, p, "mixed")
    rows = [0, 1, 2, 600, n - 1]
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, p, rows=rows)
    assert row_errors(a, y, ref, rows).max() <= TOL["mixed"]
    assert plan.report()["n_fallback"] == 0


def test_forced_fallback_matches_oracle(sm):
    a = wl.overlap_uniform(n=1500)
    plan, y = run(sm, a, 2, "mixed", resid_tol=1e-300)
    rep = plan.report()
    assert rep["n_fallback"] == a.n
    rows = sample_rows(a, 80)
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, 2, rows=rows)
    assert row_errors(a, y, ref, rows).max() <= 1e-10


def test_not_spd_rows_are_nan_and_reported(sm):
    a = wl.overlap_small(n=500)
    vals = a.vals.copy()
    j = 17
    d = a.rowptr[j] + int(np.nonzero(a.colind[a.rowptr[j]:a.rowptr[j + 1]] == j)[0][0])
    vals[d] = -50.0
    plan = sm.submat_plan(a.rowptr, a.colind, 2)
    v = torch.tensor(vals, device="cuda")
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_invroot(plan, v, sync=True)
    assert ei.value.name == "SUBMAT_ENOTSPD"
    y = sm.submat_invroot(plan, v).cpu().numpy()
    torch.cuda.synchronize()
    bad = [r for r in range(a.n) if np.isnan(y[a.rowptr[r]:a.rowptr[r + 1]]).any()]
    assert j in bad
    # every submatrix containing row/column 17 is affected; all others are finite & right
    affected = {r for r in range(a.n) if 17 in a.colind[a.rowptr[r]:a.rowptr[r + 1]]}
    assert set(bad) <= affected
    good = [r for r in range(a.n) if r not in affected][:60]
    ref = oracle.invroot(a.rowptr, a.colind, vals, 2, rows=good)
    assert row_errors(a, y, ref, good).max() <= 1e-6


def test_nan_input_reported(sm):
    a = wl.overlap_small(n=300)
    vals = a.vals.copy()
    vals[5] = np.nan
    plan = sm.submat_plan(a.rowptr, a.colind, 2)
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_invroot(plan, torch.tensor(vals, device="cuda"), sync=True)
    assert ei.value.name == "SUBMAT_ENOTSPD"


def test_graph_and_stream_paths_agree(sm):
    a = wl.overlap_uniform(n=2000)
    v = torch.tensor(a.vals, device="cuda")
    p1 = sm.submat_plan(a.rowptr, a.colind, 2, use_graph=True)
    p2 = sm.submat_plan(a.rowptr, a.colind, 2, use_graph=False)
    y1 = sm.submat_invroot(p1, v)
    y1b = sm.submat_invroot(p1, v)           # graph replay
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        y2 = sm.submat_invroot(p2, v, stream=s)
    s.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(y1, y1b)
    assert torch.equal(y1, y2)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_repeat_runs_bitwise_equal(sm, precision):
    """Every reduction that steers the iteration (norms, maxima) is taken in a fixed order,
    so repeated calls give identical bits (orders 40..250: ragged tiles and mirror images)."""
    for a in (wl.overlap_uniform(n=1500), wl.overlap_small(n=800)):
        v = torch.tensor(a.vals, device="cuda")
        plan = sm.submat_plan(a.rowptr, a.colind, 2, precision=precision, use_graph=False)
        ys = [sm.submat_invroot(plan, v, sync=True) for _ in range(3)]
        for y in ys[1:]:
            assert torch.equal(ys[0], y)


def test_device_pattern_input(sm):
    a = wl.overlap_small(n=700)
    rp = torch.tensor(a.rowptr, device="cuda")
    ci = torch.tensor(a.colind, device="cuda")
    plan = sm.submat_plan(rp, ci, 2)
    m, pos = plan.rows()
    mo, po = oracle.plan(a.rowptr, a.colind)
    np.testing.assert_array_equal(m, mo)
    np.testing.assert_array_equal(pos, po)


def test_host_buffers_match_device_path(sm):
    """submat_invroot_host (host arrays in and out, copies inside the call) gives the device
    path's bits, from numpy arrays and from pinned tensors, and meets the bar."""
    a = wl.overlap_uniform(n=600, kappa=1e3)
    plan = sm.submat_plan(a.rowptr, a.colind, 2)
    v = torch.tensor(a.vals, device="cuda")
    yd = sm.submat_invroot(plan, v, sync=True).cpu().numpy()
    yh = plan.invroot_host(a.vals)
    assert np.array_equal(yh, yd)
    hin = torch.tensor(a.vals).pin_memory()
    hout = torch.empty(a.nnz, dtype=torch.float64).pin_memory()
    plan.invroot_host(hin, hout)
    assert np.array_equal(hout.numpy(), yd)
    rows = list(range(0, a.n, 5))
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, 2, rows=rows)
    assert row_errors(a, yh, ref, rows).max() <= TOL["mixed"]


def test_invalid_calls(sm):
    a = wl.overlap_small(n=200)
    plan = sm.submat_plan(a.rowptr, a.colind, 2)
    v = torch.tensor(a.vals, device="cuda")
    st = plan._lib.submat_invroot(plan._h, v.data_ptr(), v.data_ptr(), None, 1)
    assert sm.STATUS[st] == "SUBMAT_EINVAL"           # vals_out overlapping vals_in
    nofwd = sm.submat_plan(a.rowptr, a.colind, 2)
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_invroot_backward(nofwd, v)
    assert ei.value.name == "SUBMAT_ENOFWD"
    # non-symmetric pattern / missing diagonal / unsorted
    dense = np.eye(4) * 2
    dense[0, 1] = 0.5
    c = wl.dense_to_csr(dense)
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_plan(c.rowptr, c.colind, 2)
    assert ei.value.name == "SUBMAT_ENOTSYM"
    keep = np.ones((3, 3), bool)
    keep[1, 1] = False
    c = wl.dense_to_csr(np.ones((3, 3)), keep=keep)
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_plan(c.rowptr, c.colind, 2)
    assert ei.value.name == "SUBMAT_ENODIAG"
    c = wl.dense_to_csr(np.ones((3, 3)) + np.eye(3))
    ci = c.colind.copy()
    ci[0], ci[1] = ci[1], ci[0]
    with pytest.raises(sm.SubmatError) as ei:
        sm.submat_plan(c.rowptr, ci, 2)
    assert ei.value.name == "SUBMAT_EINVAL"


@pytest.mark.parametrize("p", [1, 2, 3])
def test_tcgen05_and_mma_sync_engines_agree(sm, p):
    # same arithmetic on two tensor-core engines; both must meet the bar against the oracle
    a = wl.overlap_uniform(n=3000)
    rows = sample_rows(a, 60, seed=10 + p)
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, p, rows=rows)
    outs = {}
    for prec in ("mixed", "mixed_sync"):
        plan, y = run(sm, a, p, prec)
        assert row_errors(a, y, ref, rows).max() <= TOL["mixed"]
        outs[prec] = y
    assert row_errors(a, outs["mixed"], outs["mixed_sync"], range(a.n)).max() <= 1e-6


# ---------------------------------------------------------------------------
# Positive p-th roots (Sec. 4.2; root_sign = +1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_positive_root_small_all_rows(sm, precision):
    a = wl.overlap_small()
    plan, y = run(sm, a, 2, precision, root_sign=1)
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, 2, sign=1)
    assert row_errors(a, y, ref, range(a.n)).max() <= TOL[precision]


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_positive_root_uniform_sampled(sm, p, precision):
    a = wl.overlap_uniform(n=4096)
    plan, y = run(sm, a, p, precision, root_sign=1)
    rows = sample_rows(a, 100, seed=10 + p)
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, p, rows=rows, sign=1)
    assert row_errors(a, y, ref, rows).max() <= TOL[precision]
    assert plan.report()["n_fallback"] == 0


def test_positive_root_dense_pattern_is_full_root(sm):
    import scipy.linalg as sl
    rng = np.random.default_rng(19)
    b = rng.standard_normal((90, 90))
    dense = b @ b.T / 90 + 0.3 * np.eye(90)
    a = wl.dense_to_csr(dense, keep=np.ones((90, 90), dtype=bool))
    for p in (2, 3):
        plan, y = run(sm, a, p, "mixed", root_sign=1)
        full = np.real(sl.fractional_matrix_power(dense, 1.0 / p))
        yd = oracle.to_dense(a.n, a.rowptr, a.colind, y)
        assert np.abs(yd - full.T).max() / np.abs(full).max() < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shards_reproduce_the_whole(sm, precision):
    """Plans for the shards of a row partition (one GPU each in a multi-GPU run; here the
    shards run one after another) write disjoint row segments that together equal the
    unsharded forward bit for bit, and their backward contributions add up to the full
    gradient."""
    a = wl.overlap_uniform(n=1200, kappa=1e3)
    v = torch.tensor(a.vals, device="cuda")
    w = torch.tensor(wl.random_on_pattern(a, seed=9), device="cuda")
    full = sm.submat_plan(a.rowptr, a.colind, 2, precision=precision)
    y = sm.submat_invroot(full, v)
    g = sm.submat_invroot_backward(full, w)
    ys = torch.full_like(v, float("nan"))
    gs = torch.zeros_like(v)
    for rank in range(3):
        b, e = sm.shard_rows(a.rowptr, 3, rank)
        plan = sm.submat_plan(a.rowptr, a.colind, 2, precision=precision, shard=(rank, 3))
        assert plan.report()["n_rows"] == e - b
        sm.submat_invroot(plan, v, ys)
        gs += sm.submat_invroot_backward(plan, w)
    torch.cuda.synchronize()
    assert torch.equal(ys, y)
    assert (gs - g).abs().max().item() <= 1e-12 * g.abs().max().item()


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("sign", [-1, 1])
def test_taylor_finish_without_products(sm, p, sign):
    """Submatrices already within the stopping distance of I (||M_0 - I||_F <= 0.05) take
    no GEMM iteration: the Taylor finish on the carried column alone gives the root."""
    rng = np.random.default_rng(20 + p)
    n = 300
    off = rng.uniform(-1e-3, 1e-3, n - 1)
    a = wl.dense_to_csr(np.eye(n) + np.diag(off, 1) + np.diag(off, -1))
    plan = sm.submat_plan(a.rowptr, a.colind, p, precision="mixed", root_sign=sign)
    y = sm.submat_invroot(plan, torch.tensor(a.vals, device="cuda"), sync=True).cpu().numpy()
    assert plan.report()["iters_max"] == 0
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, p, sign=sign)
    assert row_errors(a, y, ref, range(a.n)).max() <= TOL["mixed"]
