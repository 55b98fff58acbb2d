"""Tune the mixed-precision forward's size buckets on the GPU at hand and write them into
``csrc/engine_table.h`` (rebuild the library afterwards).

For every row order m in the candidate list, a block-diagonal workload whose rows all have
order m (``workloads.block_diagonal_spd``, enough rows to fill every SM several times) is run
through each engine that can take it: the small engine (working set in shared memory, 16 x 8
warp tiles), the mma.sync engine (64 x 64 tiles) and the tcgen05 engine (128 x 96 tiles in
tensor memory).  The time per forward is the median of ``--steps`` CUDA-event timed calls
after ``--warmup`` untimed ones.  The small engine takes the orders from 1 up to the largest
m at which it is the fastest engine with every smaller candidate also won by it; the mma.sync
bucket continues from there the same way; larger rows take the tcgen05 engine.

    python -m paper_1710_10899_gb300.tune [--steps 5] [--warmup 2] [--out PATH]
"""
from __future__ import annotations

import argparse
import os
import statistics
import sys
import time

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CANDIDATES = [8, 16, 24, 32, 48, 64, 96, 128]
ENGINES = {"small": dict(small_max_m=32, sync_max_m=0),
           "sync": dict(small_max_m=0, sync_max_m=1536),
           "tcgen05": dict(small_max_m=0, sync_max_m=0)}


def time_forward(sm, a, p, opts, steps, warmup):
    import torch
    plan = sm.submat_plan(a.rowptr, a.colind, p, precision="mixed", **opts)
    v = torch.tensor(a.vals, device="cuda")
    out = torch.empty_like(v)
    for _ in range(warmup):
        sm.submat_invroot(plan, v, out)
    torch.cuda.synchronize()
    ms = []
    stream = torch.cuda.current_stream()
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sm.submat_invroot(plan, v, out)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def choose(times):
    """(small_max_m, sync_max_m) from {m: {engine: ms}} as described in the module doc."""
    small_max = 0
    for m in sorted(times):
        t = times[m]
        if "small" in t and t["small"] <= min(t.values()):
            small_max = m
        else:
            break
    sync_max = 0
    for m in sorted(times):
        if m <= small_max:
            continue
        t = times[m]
        if t["sync"] <= min(t.values()):
            sync_max = m
        else:
            break
    return small_max, sync_max


def write_header(path, small_max, sync_max, times, rows_per_case, gpu):
    lines = [
        "// Size buckets of the mixed-precision forward: which engine takes a row of order m.",
        "// Written by paper_1710_10899_gb300/tune.py from forward times measured on a GB300 (the",
        "// measurements are listed below); rows of order m <= kTunedSmallMaxM go to the small engine",
        "// (working set in shared memory, 16 x 8 warp tiles of mma.sync), rows with",
        "// kTunedSmallMaxM < m <= kTunedSyncMaxM to the mma.sync engine (64 x 64 tiles, cp.async",
        "// pipeline), the rest to the tcgen05 engine (128 x 96 tiles in TMEM, TMA pipeline).",
        f"// Device: {gpu}; p = 2; {rows_per_case} rows of one order per case; ms per forward",
        "// (median):",
        "//     m   " + "".join(f"{e:>10}" for e in ENGINES),
    ]
    for m in sorted(times):
        lines.append(f"//  {m:4d}   " + "".join(
            f"{times[m][e]:10.3f}" if e in times[m] else f"{'-':>10}" for e in ENGINES))
    lines += ["#pragma once", "namespace submat {",
              f"constexpr int kTunedSmallMaxM = {small_max};",
              f"constexpr int kTunedSyncMaxM = {sync_max};",
              "}  // namespace submat", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--rows", type=int, default=152 * 2 * 24)
    ap.add_argument("--out", default=os.path.join(PKG, "csrc", "engine_table.h"))
    args = ap.parse_args()
    import torch
    import workloads as wl
    import paper_1710_10899_gb300 as sm
    sm.load_library()
    times = {}
    for m in CANDIDATES:
        a = wl.block_diagonal_spd(max(1, args.rows // m), m, seed=m)
        times[m] = {}
        for name, opts in ENGINES.items():
            if name == "small" and m > sm.SUBMAT_SMALL_MAX_M:
                continue
            t0 = time.perf_counter()
            times[m][name] = time_forward(sm, a, 2, opts, args.steps, args.warmup)
            sys.stderr.write(f"m={m:4d} {name:8s} {times[m][name]:9.3f} ms "
                             f"({time.perf_counter() - t0:.1f} s)\n")
    small_max, sync_max = choose(times)
    write_header(args.out, small_max, sync_max, times, args.rows,
                 torch.cuda.get_device_name(0))
    print(f"small_max_m={small_max} sync_max_m={sync_max} -> {args.out}")


if __name__ == "__main__":
    main()
