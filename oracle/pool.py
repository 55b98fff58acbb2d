"""Row-parallel evaluation of the FP64 oracle on the host cores (test infrastructure only).

The submatrix method's rows are independent (Sec. 3: every column j needs only S_j), so the
oracle's per-row functions can run in worker processes over disjoint row sets.  This module
only distributes rows and gathers the results: every value is computed by
the functions of ``oracle/submatrix.py`` as they stand, with no change to its arithmetic.  Only ``tests/`` and
``bench.py``'s oracle legs use it.

Start method: ``"fork"`` shares the matrix with the workers without copying it, but must be
used before the calling process makes its first CUDA call (a process forked after that can
hang); ``"spawn"`` is safe at any time and pickles the arrays to each worker once.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from .submatrix import grad as _grad, row_segment as _row_segment

_STATE: dict = {}


def _init(state):
    _STATE.clear()
    _STATE.update(state)


def _fwd_chunk(rows):
    s = _STATE
    segs = [_row_segment(s["rowptr"], s["colind"], s["vals"], s["p"], int(j), s["sign"])
            for j in rows]
    return rows, (np.concatenate(segs) if segs else np.zeros(0))


def _grad_chunk(rows):
    s = _STATE
    return _grad(s["rowptr"], s["colind"], s["vals"], s["p"], s["grad_out"], s["sign"],
                    rows=[int(j) for j in rows])


def default_processes():
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    return max(1, min(n, 64))


_BLAS_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _pool(state, processes, start):
    """A pool of single-threaded workers.  Spawned workers read the BLAS thread counts from
    the environment when they import numpy, so those are set to 1 around their start; a
    forked worker inherits the parent's BLAS state, so fork is only for a parent whose
    BLAS is single-threaded (set before numpy's first import)."""
    ctx = mp.get_context(start)
    if start == "fork":
        _init(state)                       # inherited by the forked workers
        return ctx.Pool(processes)
    saved = {k: os.environ.get(k) for k in _BLAS_VARS}
    for k in _BLAS_VARS:
        os.environ[k] = "1"
    try:
        return ctx.Pool(processes, initializer=_init, initargs=(state,))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _chunks(rows, processes, per_proc=4):
    rows = list(rows)
    k = max(1, min(len(rows), processes * per_proc))
    return [rows[c::k] for c in range(k)]


def invroot(rowptr, colind, vals, p, rows=None, sign=-1, processes=None, start="spawn"):
    """``oracle.invroot`` over ``rows`` (default: all) in worker processes.  Same result
    layout: the value array of length nnz, NaN outside the rows computed."""
    n = len(rowptr) - 1
    rows = range(n) if rows is None else rows
    processes = processes or default_processes()
    out = np.full(len(colind), np.nan)
    state = dict(rowptr=rowptr, colind=colind, vals=vals, p=p, sign=sign)
    with _pool(state, processes, start) as pool:
        for rs, seg in pool.imap_unordered(_fwd_chunk, _chunks(rows, processes)):
            o = 0
            for j in rs:
                m = int(rowptr[j + 1] - rowptr[j])
                out[rowptr[j]:rowptr[j + 1]] = seg[o:o + m]
                o += m
    return out


def grad(rowptr, colind, vals, p, grad_out, sign=-1, processes=None, start="spawn"):
    """``oracle.grad`` in worker processes: each sums the contributions of a row set, and the
    partial gradients are added in a fixed order."""
    n = len(rowptr) - 1
    processes = processes or default_processes()
    state = dict(rowptr=rowptr, colind=colind, vals=vals, p=p, sign=sign,
                 grad_out=np.asarray(grad_out, dtype=np.float64))
    with _pool(state, processes, start) as pool:
        parts = pool.map(_grad_chunk, _chunks(range(n), processes))
    out = np.zeros(len(colind))
    for part in parts:
        out += part
    return out
