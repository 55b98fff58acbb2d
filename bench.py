"""Benchmark of the submatrix method's hot path on one GB300 (or N replicas/shards).

A step is one whole forward over the workload: for every row j, gather S_j, compute
S_j^(-1/p) and write column pos_j back into A's pattern (Alg. 1, Sec. 3.2, Alg. 2).
Default workload: the uniform 3-D overlap matrix, n=32768 (m_j 32..255), kappa ~ 1e3, p=2,
mixed precision.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload overlap_uniform|overlap_small|overlap_clustered|overlap_grad|
                                block_overlap] [--p P] [--precision mixed|fp64]
                    [--no-fp64-compare] [--no-extras] [--extras a,b,...]

The line carries, besides the contract's keys:
  * the accuracy of every row of the result against the FP64 oracle (computed on the host
    cores before the GPU work starts; its wall time is the CPU baseline);
  * ``roofline``: the method's flops (sum over rows of k_j (p+1) 2 m_j^3, executed iteration
    counts, true orders) per launch of the dominant kernel over its CUDA-event time, against
    the measured dense BF16 (= FP16) rate; the tensor-core work the engine executes for them
    (10 FP16 slice products per product) is reported beside it as
    ``executed_tensor_tflops``;
  * ``fp64_path``: the all-FP64 GPU path on the same input (median of --fp64-steps steps)
    and its error against the oracle on every row;
  * ``extras``: the other workloads (p = 1 and 3, the positive root, the small FP64
    workload, the clustered and the block-sparse workloads, the adjoint with its atomic and
    deterministic scatters), each timed and checked against the oracle (every row, or a
    seeded sample stratified by row size), and the CG solves of Sec. 4.4 on the stand-ins
    for its matrices, plain and preconditioned with the method's result.

With N > 1 (torchrun) the workload is built N times larger (same recipe, n x N rows) and
its rows are sharded across ranks (Sec. 6.1.1: every rank holds the whole matrix and
computes a contiguous, cost-balanced range of rows; no data-path collective), so the work
per GPU stays that of the 1-GPU workload (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

# The oracle runs in single-threaded worker processes forked from this one: pin the BLAS
# pools to one thread before numpy is first imported.
for _k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_k] = "1"

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "submatrices/s & TFLOP/s for sparse A^(-1/p) at rel.err<=1e-6 vs FP64 path, % peak"
UNIT = "submatrices/s"
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
FP64_NOMINAL_TFLOPS = 1.25          # GB300 FP64 (CUDA cores), nominal
DTYPE_MIXED = "f16x4-slices/f32acc-per-level+f64"

# The extra workloads of the default run: (name, workload, p, precision, root sign, rows
# checked against the oracle (0 = every row), warm-up steps, timed steps).
EXTRAS = [
    ("uniform_p1", "overlap_uniform", 1, "mixed", -1, 1024, 3, 5),
    ("uniform_p3", "overlap_uniform", 3, "mixed", -1, 1024, 3, 5),
    ("uniform_p2_positive_root", "overlap_uniform", 2, "mixed", +1, 1024, 3, 5),
    ("small_fp64", "overlap_small", 2, "fp64", -1, 0, 3, 5),
    ("small_mixed", "overlap_small", 2, "mixed", -1, 0, 3, 5),
    ("clustered", "overlap_clustered", 2, "mixed", -1, 512, 1, 3),
    ("block", "block_overlap", 2, "mixed", -1, 128, 1, 1),
    ("backward", "overlap_grad", 2, "mixed", -1, 0, 1, 3),
    ("cg", "cg_standins", 2, "mixed", -1, 0, 1, 3),
]
CG_STANDINS = (("laplace2d_aniso(nx=64,eps=0.01)", "laplace2d_aniso", {}),
               ("jump3d(nx=16,contrast=1e4)", "jump3d", {}),
               ("overlap_uniform(n=4096,kappa=1e5)", "overlap_uniform", {"n": 4096, "kappa": 1e5}))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="overlap_uniform")
    ap.add_argument("--p", type=int, default=2)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--extras", default="",
                    help="comma-separated subset of the extra workloads (default: all)")
    ap.add_argument("--oracle-seconds", type=float, default=20.0,
                    help="reference arm: single-thread seconds of oracle work per step")
    ap.add_argument("--n", "--rows", dest="n", type=int, default=0,
                    help="scale the workload down to n rows (under torchrun use --rows: "
                         "its launcher takes --n for one of its own options)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def log(msg):
    sys.stderr.write(f"[bench {time.strftime('%H:%M:%S')}] {msg}\n")
    sys.stderr.flush()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------------------
# oracle (CPU baseline, accuracy reference, reference arm); run before any CUDA call
# ----------------------------------------------------------------------------------------
_W = {}


def _oracle_init(rowptr, colind, vals, p, route="eig"):
    _W.update(rowptr=rowptr, colind=colind, vals=vals, p=p, route=route)


def _oracle_rows(rows):
    import oracle
    if _W.get("route") == "lu":        # the paper's p = 1 route: LU inversion per submatrix
        oracle.invroot_lu(_W["rowptr"], _W["colind"], _W["vals"], rows=rows)
    else:
        oracle.invroot(_W["rowptr"], _W["colind"], _W["vals"], _W["p"], rows=rows)
    return len(rows)


def time_oracle_sampled(a, p, seconds, seed=3, steps=1, warmup=0, route="eig"):
    """The reference arm: the oracle as it stands, one single-threaded process per host core.
    Each step is a row sample sized for about ``seconds`` of single-thread CPU work
    (consecutive slices of one seeded permutation); ``warmup`` untimed steps, then ``steps``
    timed ones.  Returns (rows/s, cores, rows per step, mean wall s per timed step, sample
    description).  ``route="lu"`` (p = 1 only) times the paper's LU inversion instead."""
    import multiprocessing as mp
    import numpy as np
    import oracle
    m = a.row_sizes()
    rng = np.random.default_rng(seed)
    perm = rng.permutation(a.n)
    t0 = time.perf_counter()
    k0 = 0
    while time.perf_counter() - t0 < 0.5 and k0 < a.n:            # calibrate (one thread)
        if route == "lu":
            oracle.invroot_lu(a.rowptr, a.colind, a.vals, rows=[int(perm[k0])])
        else:
            oracle.row_segment(a.rowptr, a.colind, a.vals, p, int(perm[k0]))
        k0 += 1
    per_row = (time.perf_counter() - t0) / max(k0, 1)
    cores = min(host_cores(), 64)
    k = int(min(a.n, max(cores, seconds / per_row)))          # rows per step

    def step_chunks(i):
        rows = [int(r) for r in perm[(np.arange(k) + i * k) % a.n]]
        chunks = [rows[c::cores * 4] for c in range(cores * 4)]
        return rows, [c for c in chunks if c]

    _oracle_init(a.rowptr, a.colind, a.vals, p, route)   # inherited by the forked workers
    ctx = mp.get_context("fork")
    done, dt, msum = 0, 0.0, 0.0
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_rows, [[int(perm[0])]] * cores)     # start the workers
        for i in range(warmup):
            pool.map(_oracle_rows, step_chunks(i)[1])
        for i in range(warmup, warmup + max(steps, 1)):
            rows, chunks = step_chunks(i)
            t0 = time.perf_counter()
            done += sum(pool.map(_oracle_rows, chunks))
            dt += time.perf_counter() - t0
            msum += float(m[rows].sum())
    nst = max(steps, 1)
    sample = (f"{nst} timed step(s) after {warmup} untimed, {k} of {a.n} rows each "
              f"(slices of a seeded permutation, seed {seed}), mean m {msum / done:.1f}, "
              f"{dt:.2f} s wall on {cores} processes")
    return done / dt, cores, k, dt / nst, sample


def oracle_values(a, p, rows=None, sign=-1):
    """The oracle's values for ``rows`` (None: every row) on the host cores (forked pool;
    called before this process makes any CUDA call).  Returns (values, wall seconds)."""
    import oracle
    t0 = time.perf_counter()
    ref = oracle.pool.invroot(a.rowptr, a.colind, a.vals, p, rows=rows, sign=sign,
                              processes=min(host_cores(), 64), start="fork")
    return ref, time.perf_counter() - t0


def row_errors(a, y, ref, rows=None):
    """Per-row ||y_j - ref_j|| / ||ref_j|| over ``rows`` (None: all rows)."""
    import numpy as np
    rp = a.rowptr.astype(np.int64)
    if rows is None:
        d2 = np.add.reduceat((y - ref) ** 2, rp[:-1])
        r2 = np.add.reduceat(ref ** 2, rp[:-1])
        return np.sqrt(d2 / r2)
    out = []
    for j in rows:
        s = slice(rp[j], rp[j + 1])
        out.append(float(np.linalg.norm(y[s] - ref[s]) / np.linalg.norm(ref[s])))
    return np.array(out)


# ----------------------------------------------------------------------------------------
def make_workload(name, n=0, scale=1):
    """The named workload with n rows (0: its default size), n x scale rows in all."""
    import inspect
    import workloads as wl
    if name not in wl.WORKLOADS:
        raise SystemExit(f"unknown workload {name}")
    fn = wl.WORKLOADS[name]
    if name == "block_overlap":                     # n rows = 13 functions per atom
        atoms = n // 13 if n > 0 else inspect.signature(fn).parameters["atoms"].default
        return wl.block_overlap(atoms=max(1, atoms * scale))
    if n <= 0 and scale == 1:
        return fn()
    if n <= 0:
        n = inspect.signature(fn).parameters["n"].default
    return fn(n=n * scale)


def describe(name, a, p, sign=-1):
    root = "A^(-1/p)" if sign < 0 else "A^(1/p)"
    return f"{name}(n={a.n},nnz={a.nnz},p={p}{'' if sign < 0 else ',' + root})"


def clocks_start():
    try:
        f = open(os.path.join(ROOT, "_clocks.csv"), "w")
        proc = subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=f, stderr=subprocess.DEVNULL)
        return proc, f
    except Exception:
        return None, None


def clocks_stop(proc, f, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    f.close()
    path = os.path.join(ROOT, "_clocks.csv")
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != gpu_index:
            continue
        try:
            sm.append(float(parts[1]))
            mx = max(mx, float(parts[2]))
        except ValueError:
            continue
        for nme, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nme)
    os.remove(path)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


def traffic_for(kernel_src):
    """DRAM bytes per launch of the main kernel from the committed ncu summary, if the
    kernel source is unchanged since it was captured (else None)."""
    path = os.path.join(ROOT, "profiles", "fwd_mixed_kernel_traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    sha = hashlib.sha256(open(os.path.join(ROOT, kernel_src), "rb").read()).hexdigest()
    ent = rec.get(kernel_src)
    if not ent or ent.get("sha256") != sha:
        return None
    return ent.get("dram_bytes_per_launch")


def fp32_alu_peak_tflops(sm_mhz):
    """FP32 FMA peak of GB300's CUDA cores: 152 SMs x 128 lanes x 2 flops per clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# ----------------------------------------------------------------------------------------
# GPU timing helpers
# ----------------------------------------------------------------------------------------
def timed_forward(sm, plan, vals, out, flush, steps, warmup):
    """``warmup`` untimed forwards, then ``steps`` timed ones (L2 flushed before each, not
    timed), CUDA events on the launching stream.  Returns per-step ms and the reports."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        sm.submat_invroot(plan, vals, out)
    torch.cuda.synchronize()
    ms, reps = [], []
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sm.submat_invroot(plan, vals, out)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        reps.append(plan.report())
    return ms, reps


def roofline_mixed(reps, pk, pk_kind):
    """Roofline of fwd_mixed_kernel: the method's flops per launch over the kernel's mean
    CUDA-event time, against the measured dense BF16 (= FP16) sustained rate."""
    kern_ms = statistics.mean(r["ms_kernel"] for r in reps)
    alg = statistics.mean(r["flops_alg"] for r in reps)
    executed = statistics.mean(r["flops_tensor"] for r in reps)
    peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    achieved = alg / (kern_ms / 1e3) / 1e12
    return {"bound": "tensor", "kernel": "fwd_mixed_kernel", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_kind": f"{pk_kind} bf16 dense sustained (FP16 rate = BF16 rate)",
            "flops_per_launch": alg, "ms_kernel": kern_ms,
            "work": "sum over rows of k_j (p+1) 2 m_j^3 (executed iterations, true orders)",
            "executed_tensor_tflops": executed / (kern_ms / 1e3) / 1e12,
            "executed_tensor_frac": executed / (kern_ms / 1e3) / 1e12 / peak,
            "executed_work": "10 FP16 slice products x 2 m_j^3 per executed GEMM"}


def roofline_fp64(reps):
    kern_ms = statistics.mean(r["ms_kernel"] for r in reps)
    alg = statistics.mean(r["flops_alg"] for r in reps)
    achieved = alg / (kern_ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": "fwd_fp64_kernel", "achieved": achieved,
            "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_NOMINAL_TFLOPS, "peak_kind": "nominal FP64 rate",
            "flops_per_launch": alg, "ms_kernel": kern_ms, "traffic": None,
            "work": "sum over rows of k_j (p+1) 2 m_j^3 (executed iterations, true orders)"}


def run_extra(sm, spec, a, ref, rows_checked, flush, pk, pk_kind, clocks_mhz):
    """One extra workload: plan, warm-up, timed forwards (median), accuracy vs the oracle."""
    import numpy as np
    import torch
    name, wname, p, prec, sign, _, warm, steps = spec
    plan = sm.submat_plan(a.rowptr, a.colind, p, precision=prec, root_sign=sign)
    vals = torch.tensor(a.vals, device="cuda")
    out = torch.empty_like(vals)
    ms, reps = timed_forward(sm, plan, vals, out, flush, steps, warm)
    med = statistics.median(ms)
    y = out.cpu().numpy()
    err = row_errors(a, y, ref, rows_checked)
    rec = {"workload": describe(wname, a, p, sign), "precision": prec,
           "value": a.n / (med / 1e3), "unit": UNIT, "ms_per_step_median": med,
           "steps": steps, "warmup": warm,
           "max_row_rel_err_vs_oracle": float(err.max()),
           "rows_checked": "all" if rows_checked is None else int(len(rows_checked)),
           "tol": 1e-10 if prec == "fp64" else 1e-6,
           "fallback_rows": int(reps[-1]["n_fallback"]),
           "iters_mean": reps[-1]["iters_sum"] / max(1, a.n),
           "roofline": roofline_fp64(reps) if prec == "fp64" else roofline_mixed(reps, pk, pk_kind)}
    if rows_checked is not None:
        rec["rows_sample"] = "seeded (seed 3) sample stratified by row size, incl. the " \
                             "smallest and largest rows"
    if name == "backward":
        rec.update(backward_block(sm, plan, a, vals, flush, steps, warm, clocks_mhz))
    del plan
    return rec


def backward_block(sm, plan, a, vals, flush, steps, warm, clocks_mhz):
    """The adjoint on the differentiation workload: L = sum(W * Y), W ~ N(0,1) on the
    pattern (seed 1); timed backward calls (median) and the gradient against the oracle's
    over every stored entry (computed before the GPU work)."""
    import numpy as np
    import torch
    import workloads as wl
    w = torch.tensor(wl.random_on_pattern(a, seed=1), device="cuda")
    sm.submat_invroot(plan, vals)
    ms, g = time_backward(sm, plan, w, flush, steps, warm)
    med = statistics.median(ms)
    gref = _PRE["grad_ref"]
    gh = g.cpu().numpy()
    # the deterministic (atomic-free) scatter: per-row gradients in waves, summed per entry
    # in a fixed order
    pdet = sm.submat_plan(a.rowptr, a.colind, 2, grad_deterministic=True)
    sm.submat_invroot(pdet, vals)
    ms_det, g_det = time_backward(sm, pdet, w, flush, steps, warm)
    g_det2 = sm.submat_invroot_backward(pdet, w)
    gd = g_det.cpu().numpy()
    det = {"ms_per_call_median": statistics.median(ms_det),
           "value": a.n / (statistics.median(ms_det) / 1e3), "unit": UNIT,
           "grad_rel_err_vs_oracle": float(np.linalg.norm(gd - gref) / np.linalg.norm(gref)),
           "bitwise_repeatable": bool(torch.equal(g_det, g_det2)),
           "max_abs_diff_vs_atomic_rel_to_max": float(np.abs(gd - gh).max() / np.abs(gh).max())}
    del pdet
    m = a.row_sizes().astype(np.float64)
    work = float((16.0 * m ** 3).sum())
    mhz = clocks_mhz or 2070.0
    peak = fp32_alu_peak_tflops(mhz)
    achieved = work / (med / 1e3) / 1e12
    return {"backward": {
        "ms_per_call_median": med, "value": a.n / (med / 1e3), "unit": UNIT,
        "grad_rel_err_vs_oracle": float(np.linalg.norm(gh - gref) / np.linalg.norm(gref)),
        "grad_max_abs_err_rel_to_max": float(np.abs(gh - gref).max() / np.abs(gref).max()),
        "tol": 1e-10,
        "roofline": {"bound": "alu", "kernel": "backward_kernel", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_kind": f"FP32 FMA rate at {mhz:.0f} MHz (152 SMs x 128 lanes x 2)",
                     "work": "16 m_j^3 per row (Jacobi sweeps and eigenvector products "
                             "counted as FP64-equivalent flops, executed in double-float "
                             "FP32 arithmetic)"},
        "deterministic": det}}


def time_backward(sm, plan, w, flush, steps, warm):
    """``warm`` untimed and ``steps`` CUDA-event timed backward calls (L2 flushed before
    each, not timed).  Returns (per-call ms, last gradient)."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        sm.submat_invroot_backward(plan, w)
    torch.cuda.synchronize()
    ms, g = [], None
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g = sm.submat_invroot_backward(plan, w)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms, g


def cg_block(sm, spec, flush):
    """The preconditioning application (Sec. 4.4) on the stand-ins for the section's
    matrices: CG on A x = ones (threshold 1e-6), plain and with K = the p = 2 result of the
    method (K ~ A^(-1/2)); per matrix the steps, the CUDA-event time of a solve (median of
    ``steps`` after ``warm`` untimed ones; the solver's host loop reads two scalars per step)
    and of the forward that makes K."""
    import torch
    _, _, p, prec, _, _, warm, steps = spec
    import workloads as wl
    out = {}
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ms, res = [], None
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms), res

    for label, fname, kw in CG_STANDINS:
        a = wl.WORKLOADS[fname](**kw) if fname in wl.WORKLOADS else getattr(wl, fname)(**kw)
        plan = sm.submat_plan(a.rowptr, a.colind, p, precision=prec)
        v = torch.tensor(a.vals, device="cuda")
        k = torch.empty_like(v)
        ms_fwd, _ = timed(lambda: sm.submat_invroot(plan, v, k))
        ms_plain, (_, it_plain, rel_plain) = timed(lambda: sm.submat_pcg(plan, v))
        ms_k, (_, it_k, rel_k) = timed(lambda: sm.submat_pcg(plan, v, vals_k=k))
        out[label] = {"n": a.n, "nnz": a.nnz, "steps_plain": it_plain, "steps_k": it_k,
                      "rel_resid_plain": rel_plain, "rel_resid_k": rel_k,
                      "ms_solve_plain": ms_plain, "ms_solve_k": ms_k,
                      "ms_per_step_plain": ms_plain / max(1, it_plain),
                      "ms_per_step_k": ms_k / max(1, it_k),
                      "ms_forward_k": ms_fwd, "k_precision": prec}
        del plan
    return {"workload": "CG stand-ins for Sec. 4.4 (b = ones, threshold 1e-6)",
            "steps": steps, "warmup": warm, "solves": out}


_PRE = {}


# ----------------------------------------------------------------------------------------
def main():
    args = parse()
    rank, world, local = dist_env()
    import numpy as np

    log(f"generating {args.workload}")
    a = make_workload(args.workload, args.n, scale=world)
    p = args.p
    log(f"n={a.n} nnz={a.nnz}")
    workload_name = describe(args.workload, a, p)

    if args.impl == "reference":
        if rank != 0:
            return
        v, cores, k, wall, sample = time_oracle_sampled(a, p, args.oracle_seconds,
                                                        steps=args.steps, warmup=args.warmup)
        extra = {}
        if p == 1:          # the paper's own p = 1 route (LU inversion), reported beside it
            vl, cl, _, _, sl = time_oracle_sampled(a, p, args.oracle_seconds, steps=args.steps,
                                                   warmup=args.warmup, route="lu")
            extra["paper_lu_p1"] = {"value": vl, "unit": UNIT, "cores": cl, "sample": sl}
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall,
            "step_rows": k, "ms_full_workload_extrapolated": 1e3 * a.n / v,
            "step_note": (f"a step is a sample of {k} of the workload's {a.n} rows; "
                          "ms_full_workload_extrapolated scales the sampled rate to all rows"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            **extra,
        }))
        return

    # ---- host phase: the oracle on the host cores, before any CUDA call ------------------
    do_extras = (rank == 0 and world == 1 and not args.no_extras)
    extras = []
    if do_extras:
        want = set(x for x in args.extras.split(",") if x) or None
        extras = [e for e in EXTRAS if want is None or e[0] in want]
    cpu_base, ref_all = None, None
    if rank == 0 and world == 1:
        log("oracle on every row (CPU baseline)")
        ref_all, dt = oracle_values(a, p)
        cores = min(host_cores(), 64)
        cpu_base = {"value": a.n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                    "sample": f"the whole workload: all {a.n} rows, one pass, {dt:.2f} s wall "
                              f"on {cores} single-threaded processes"}
        log(f"oracle: {a.n / dt:.1f} rows/s on {cores} cores")
    extra_inputs = {}
    import workloads as wl
    for spec in extras:
        name, wname, ep, prec, sign, nrows, _, _ = spec
        if name == "cg":                          # CG solves: no forward oracle needed
            extra_inputs[name] = (None, None, None)
            continue
        key = (wname, args.n if wname == args.workload else 0)
        if wname == args.workload:
            ea = a
        elif key in _PRE:
            ea = _PRE[key]
        else:
            log(f"generating {wname}")
            ea = make_workload(wname, 0)
            _PRE[key] = ea
        rows = None if nrows == 0 else wl.stratified_rows(ea.row_sizes(), nrows, seed=3)
        log(f"oracle for {name}: {'all' if rows is None else len(rows)} rows")
        if ea is a and ep == p and sign == -1 and rows is None:
            ref = ref_all
        else:
            ref, _ = oracle_values(ea, ep, rows=rows, sign=sign)
        if name == "backward":
            import oracle
            w = wl.random_on_pattern(ea, seed=1)
            log("oracle gradient (every row)")
            _PRE["grad_ref"] = oracle.pool.grad(ea.rowptr, ea.colind, ea.vals, ep, w,
                                                processes=min(host_cores(), 64), start="fork")
        extra_inputs[name] = (ea, ref, rows)

    import torch
    import paper_1710_10899_gb300 as sm
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    log("plan")
    plan = sm.submat_plan(a.rowptr, a.colind, p, precision=args.precision, shard=(rank, world))
    row_b, row_e = sm.shard_rows(a.rowptr, world, rank)
    launches_per_step = plan.engine_launches()
    log("warm-up")
    vals = torch.tensor(a.vals, device=dev)
    out = torch.empty_like(vals)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        sm.submat_invroot(plan, vals, out)
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed before each (flush not timed) --------------
    ms_steps, reps = [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    cproc, cf = clocks_start()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sm.submat_invroot(plan, vals, out)
        e1.record(stream)
        e1.synchronize()
        ms_steps.append(e0.elapsed_time(e1))
        reps.append(plan.report())
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clocks_stop(cproc, cf, local)
    total_ms = sum(ms_steps)
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    rows_total = a.n                               # all shards together
    value = rows_total / (ms_per_step / 1e3)
    log(f"timed: {ms_per_step:.2f} ms/step")

    # ---- accuracy (outside the timed region) ---------------------------------------------
    y = out.cpu().numpy()
    acc = {}
    if rank == 0 and ref_all is not None:
        err = row_errors(a, y, ref_all)
        acc = {"max_row_rel_err_vs_oracle": float(err.max()),
               "rows_checked_vs_oracle": int(a.n),
               "rows_over_tol": int((err > (1e-6 if args.precision == "mixed" else 1e-10)).sum())}
    elif rank == 0:
        import oracle
        rng = np.random.default_rng(11)
        rows = row_b + rng.choice(row_e - row_b, size=min(48, row_e - row_b), replace=False)
        ref = oracle.invroot(a.rowptr, a.colind, a.vals, p, rows=[int(j) for j in rows])
        acc = {"max_row_rel_err_vs_oracle": float(row_errors(a, y, ref, rows).max()),
               "rows_checked_vs_oracle": int(len(rows))}

    # ---- end to end through the C ABI with host buffers (pinned) ------------------------
    hin = torch.tensor(a.vals).pin_memory()
    hout = torch.empty(a.nnz, dtype=torch.float64).pin_memory()
    plan.invroot_host(hin, hout)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(max(2, args.steps // 2)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.invroot_host(hin, hout)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_step = statistics.mean(e2e_ms)
    if world > 1:
        t = torch.tensor([e2e_step], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_step = float(t.item())
    log(f"e2e: {e2e_step:.2f} ms/step")

    # ---- the all-FP64 GPU path on the same input ------------------------------------------
    fp64 = None
    if world == 1 and not args.no_fp64_compare and args.precision == "mixed":
        log(f"FP64 path (1 warm-up, median of {args.fp64_steps})")
        pl64 = sm.submat_plan(a.rowptr, a.colind, p, precision="fp64")
        o64 = torch.empty_like(vals)
        ms64, reps64 = timed_forward(sm, pl64, vals, o64, flush, max(1, args.fp64_steps), 1)
        med64 = statistics.median(ms64)
        log(f"FP64 path: {med64:.1f} ms")
        y64 = o64.cpu().numpy()
        fp64 = {"value": a.n / (med64 / 1e3), "unit": UNIT, "ms_per_step_median": med64,
                "steps": len(ms64), "warmup": 1, "ms_per_step_all": ms64,
                "roofline": roofline_fp64(reps64),
                "mixed_vs_fp64_max_row_rel_err": float(row_errors(a, y, y64).max()),
                "speedup_mixed_over_fp64": med64 / statistics.median(ms_steps)}
        if ref_all is not None:
            fp64["max_row_rel_err_vs_oracle"] = float(row_errors(a, y64, ref_all).max())
            fp64["rows_checked_vs_oracle"] = int(a.n)
        del pl64

    reps_all = reps
    if world > 1:                                   # the job's flops (all shards)
        t = torch.tensor([sum(r["flops_alg"] for r in reps)], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        flops_job = float(t.item())
    else:
        flops_job = sum(r["flops_alg"] for r in reps_all)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    pk, pk_kind = peaks()
    if args.precision == "mixed":
        roof = roofline_mixed(reps, pk, pk_kind)
        roof["traffic"] = traffic_for("paper_1710_10899_gb300/csrc/fwd_mixed.cu")
    else:
        roof = roofline_fp64(reps)

    # ---- extra workloads (1 GPU only; outside the main timed region) ----------------------
    extra_out = {}
    if extras:
        del plan
        torch.cuda.empty_cache()
        mhz = clocks["sm_mhz"] if clocks else None
        for spec in extras:
            name = spec[0]
            ea, ref, rows = extra_inputs[name]
            log(f"extra: {name}")
            try:
                if name == "cg":
                    extra_out[name] = cg_block(sm, spec, flush)
                else:
                    extra_out[name] = run_extra(sm, spec, ea, ref, rows, flush, pk, pk_kind, mhz)
            except Exception as e:                  # report, keep the main line
                extra_out[name] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_MIXED if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": workload_name, "precision": args.precision,
                   "l2": "flushed before every step (512 MB write, untimed)",
                   "parallelism": (f"rows sharded over {world} GPUs (cost-balanced contiguous "
                                   f"ranges, whole matrix on every GPU)") if world > 1 else "1 GPU"},
        "tflops_alg": (flops_job / args.steps / (ms_per_step / 1e3)) / 1e12,
        **acc,
        "fallback_rows_per_step": statistics.mean(r["n_fallback"] for r in reps),
        "iters_mean": reps[-1]["iters_sum"] / max(1, reps[-1]["n_rows"]),
        "roofline": roof,
        "e2e": {"value": rows_total / (e2e_step / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(a.nnz * 8 * world),
                "d2h_bytes_per_step": int(a.nnz * 8 * world)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if fp64 is not None:
        line["fp64_path"] = fp64
    if cpu_base is not None:
        line["cpu_baseline"] = cpu_base
    if extra_out:
        line["extras"] = extra_out
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
