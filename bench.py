"""Benchmark of the submatrix method's hot path on one GB300 (or N replicas/shards).

A step is one whole forward over the workload: for every row j, gather S_j, compute
S_j^(-1/p) and write column pos_j back into A's pattern (Alg. 1, Sec. 3.2, Alg. 2).
Default workload: the uniform 3-D overlap matrix, n=32768 (m_j 32..255), kappa ~ 1e3, p=2,
mixed precision.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload overlap_uniform|overlap_small|overlap_clustered|overlap_grad]
                    [--p P] [--precision mixed|fp64] [--no-fp64-compare]

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

# The oracle baseline runs one single-threaded process per core: pin the BLAS pools to one
# thread before numpy is first imported (the workers are forked from this process).
for _k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_k] = "1"

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "submatrices/s & TFLOP/s for sparse A^(-1/p) at rel.err<=1e-6 vs FP64 path, % peak"
UNIT = "submatrices/s"
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2


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
    ap.add_argument("--oracle-seconds", type=float, default=20.0,
                    help="single-thread seconds of oracle work per sampled step")
    ap.add_argument("--n", "--rows", dest="n", type=int, default=0,
                    help="scale the workload down to n rows (under torchrun use --rows: "
                         "its launcher takes --n for one of its own options)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm)
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


def log(msg):
    sys.stderr.write(f"[bench {time.strftime('%H:%M:%S')}] {msg}\n")
    sys.stderr.flush()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def time_oracle(a, p, seconds, seed=3, steps=1, warmup=0, route="eig"):
    """The oracle as it stands, one single-threaded process per host core.  Each step is a
    row sample sized for about ``seconds`` of single-thread CPU work (consecutive slices of
    one seeded permutation, so the steps take different rows while the matrix has enough);
    ``warmup`` untimed steps, then ``steps`` timed ones.  Returns (rows/s over the timed
    steps, cores, sample description).  The pool is forked before this process makes any
    CUDA call.  ``route="lu"`` (p = 1 only) times the paper's LU inversion instead of the
    eigendecomposition."""
    import multiprocessing as mp
    import numpy as np
    import oracle
    m = a.row_sizes()
    rng = np.random.default_rng(seed)
    perm = rng.permutation(a.n)
    # calibrate on a few rows in this process (single thread)
    t0 = time.perf_counter()
    k0 = 0
    while time.perf_counter() - t0 < 0.5 and k0 < a.n:
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
    return done / dt, cores, sample


# ----------------------------------------------------------------------------------------
def make_workload(name, p, n=0, scale=1):
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


def main():
    args = parse()
    rank, world, local = dist_env()
    import numpy as np

    log(f"generating {args.workload}")
    a = make_workload(args.workload, args.p, args.n, scale=world)
    p = args.p
    log(f"n={a.n} nnz={a.nnz}")
    workload_name = f"{args.workload}(n={a.n},nnz={a.nnz},p={p})"

    if args.impl == "reference":
        if rank != 0:
            return
        v, cores, sample = time_oracle(a, p, args.oracle_seconds, steps=args.steps,
                                       warmup=args.warmup)
        extra = {}
        if p == 1:          # the paper's own p = 1 route (LU inversion), reported beside it
            vl, cl, sl = time_oracle(a, p, args.oracle_seconds, steps=args.steps,
                                     warmup=args.warmup, route="lu")
            extra["paper_lu_p1"] = {"value": vl, "unit": UNIT, "cores": cl, "sample": sl}
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * a.n / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            **extra,
        }))
        return

    import torch
    import paper_1710_10899_gb300 as sm
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    # rows of this rank: a contiguous, cost-balanced shard of the world-times-larger matrix
    # (weak scaling: about the 1-GPU workload's rows per rank; with world == 1 all rows)
    cpu_base = None
    if rank == 0 and world == 1:
        # time the oracle before any GPU work starts the CUDA context in the pool's parent
        log("timing the oracle on the host cores")
        cpu_base = time_oracle(a, p, args.oracle_seconds)
        log(f"oracle: {cpu_base[0]:.1f} rows/s on {cpu_base[1]} cores")

    log("plan")
    plan = sm.submat_plan(a.rowptr, a.colind, p, precision=args.precision, shard=(rank, world))
    row_b, row_e = sm.shard_rows(a.rowptr, world, rank)
    log("warm-up")
    vals = torch.tensor(a.vals, device=dev)
    out = torch.empty_like(vals)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        sm.submat_invroot(plan, vals, out)
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed before each (flush not timed) --------------
    ms_steps, ms_kern, flops_t, flops_64, fallbacks = [], [], 0.0, 0.0, 0
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
        rep = plan.report()
        ms_kern.append(rep["ms_kernel"])
        flops_t += rep["flops_tensor"]
        flops_64 += rep["flops_fp64"]
        fallbacks += rep["n_fallback"]
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
    # ---- accuracy on sampled rows (outside the timed region) ----------------------------
    y = out.cpu().numpy()
    max_err = None
    if rank == 0:
        import oracle
        rng = np.random.default_rng(11)
        rows = row_b + rng.choice(row_e - row_b, size=min(48, row_e - row_b), replace=False)
        errs = []
        for j in rows:
            s = slice(a.rowptr[j], a.rowptr[j + 1])
            ref = oracle.row_segment(a.rowptr, a.colind, a.vals, p, int(j))
            errs.append(float(np.linalg.norm(y[s] - ref) / np.linalg.norm(ref)))
        max_err = max(errs)

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
    # ---- the all-FP64 GPU path on the same input (one step, for the comparison) ----------
    fp64 = None
    if world == 1 and not args.no_fp64_compare and args.precision == "mixed":
        log("FP64 path (one step)")
        pl64 = sm.submat_plan(a.rowptr, a.colind, p, precision="fp64")
        o64 = torch.empty_like(vals)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sm.submat_invroot(pl64, vals, o64)
        e1.record(stream)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1)
        log(f"FP64 path: {ms64:.1f} ms")
        r64 = pl64.report()
        d = (out - o64).cpu().numpy()
        y64 = o64.cpu().numpy()
        worst = 0.0
        for j in range(0, a.n, max(1, a.n // 4096)):
            s = slice(a.rowptr[j], a.rowptr[j + 1])
            worst = max(worst, float(np.linalg.norm(d[s]) / np.linalg.norm(y64[s])))
        fp64 = {"value": a.n / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                "tflops_fp64": r64["flops_fp64"] / (ms64 / 1e3) / 1e12,
                "mixed_vs_fp64_max_row_rel_err": worst,
                "speedup_mixed_over_fp64": ms64 / ms_per_step}
        del pl64

    if world > 1:                                   # the job's tensor flops (all shards)
        t = torch.tensor([flops_t], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        flops_job = float(t.item())
    else:
        flops_job = flops_t
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    pk, pk_kind = peaks()
    kern_ms = statistics.mean(ms_kern)
    flops_per_launch = flops_t / args.steps
    if args.precision == "mixed":
        achieved = flops_per_launch / (kern_ms / 1e3) / 1e12
        peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
        roof = {"bound": "tensor", "kernel": "fwd_mixed_kernel", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_kind": f"{pk_kind} bf16 dense sustained (FP16 rate = BF16 rate)",
                "traffic": traffic_for("paper_1710_10899_gb300/csrc/fwd_mixed.cu")}
    else:
        achieved = (flops_64 / args.steps) / (kern_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": "fwd_fp64_kernel", "achieved": achieved,
                "peak": 1.25, "unit": "TFLOP/s", "frac": achieved / 1.25,
                "peak_kind": "nominal FP64 rate", "traffic": None}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f16-pair/f32acc+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": workload_name, "precision": args.precision,
                   "l2": "flushed before every step (512 MB write, untimed)",
                   "parallelism": (f"rows sharded over {world} GPUs (cost-balanced contiguous "
                                   f"ranges, whole matrix on every GPU)") if world > 1 else "1 GPU"},
        "tflops": (flops_job / args.steps / (ms_per_step / 1e3)) / 1e12,
        # the same products counted once each (2 m^3 per GEMM instead of 15 slice products)
        "gemm_tflops": (flops_job / (15.0 if args.precision == "mixed" else 1.0)
                        / args.steps / (ms_per_step / 1e3)) / 1e12,
        "max_row_rel_err_vs_oracle_sampled": max_err,
        "fallback_rows_per_step": fallbacks / args.steps,
        "roofline": roof,
        "e2e": {"value": rows_total / (e2e_step / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(a.nnz * 8 * world),
                "d2h_bytes_per_step": int(a.nnz * 8 * world)},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
    }
    if fp64 is not None:
        line["fp64_path"] = fp64
    if cpu_base is not None:
        v, cores, sample = cpu_base
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
