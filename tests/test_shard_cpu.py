"""Row sharding across workers (Sec. 6.1.1; the N > 1 path) on the CPU: the cost-balanced
contiguous ranges of submat_shard_rows (host code of the library, no GPU), and a
world-size-2 gloo run in which each rank computes its shard's rows with the oracle and
the segments are gathered (the paper's final Gatherv), reproducing the unsharded result."""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads as wl


@pytest.fixture(scope="module")
def pkg():
    import paper_1710_10899_gb300 as p
    try:
        p.load_library()
    except OSError as e:           # the library is built by __graft_entry__.build()
        pytest.skip(f"library not built: {e}")
    return p


def _cost(a, lo, hi):
    m = np.diff(a.rowptr)[lo:hi].astype(np.float64)
    return float((m ** 3).sum())


@pytest.mark.parametrize("count", [1, 2, 3, 8])
def test_shard_rows_tile_and_balance(pkg, count):
    a = wl.overlap_uniform(n=3000, kappa=1e3)
    ranges = [pkg.shard_rows(a.rowptr, count, k) for k in range(count)]
    assert ranges[0][0] == 0 and ranges[-1][1] == a.n
    for (b0, e0), (b1, e1) in zip(ranges, ranges[1:]):
        assert e0 == b1 and b0 <= e0
    total = _cost(a, 0, a.n)
    mmax3 = float(np.diff(a.rowptr).max()) ** 3
    for b, e in ranges:        # each shard within one row's cost of an equal share
        assert abs(_cost(a, b, e) - total / count) <= mmax3 + 1e-9 * total


def test_shard_rows_invalid(pkg):
    rp = np.array([0, 1, 2], dtype=np.int32)
    for count, rank in [(0, 0), (2, 2), (2, -1)]:
        with pytest.raises(pkg.SubmatError) as ei:
            pkg.shard_rows(rp, count, rank)
        assert ei.value.name == "SUBMAT_EINVAL"


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import paper_1710_10899_gb300 as p
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a = wl.overlap_uniform(n=400, kappa=1e3)
    b, e = p.shard_rows(a.rowptr, world, rank)
    seg = oracle.invroot(a.rowptr, a.colind, a.vals, 2, rows=range(b, e))
    mine = torch.tensor(seg[a.rowptr[b]:a.rowptr[e]])
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([mine.numel()]))
    # gloo gathers equal sizes: pad to the largest segment, trim after
    top = int(max(int(t.item()) for t in sizes))
    padded = torch.zeros(top, dtype=torch.float64)
    padded[:mine.numel()] = mine
    parts = [torch.zeros(top, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, padded)
    if rank == 0:
        np.save(out, torch.cat([q[:int(t.item())] for q, t in zip(parts, sizes)]).numpy())
    dist.destroy_process_group()


def test_gloo_two_ranks_assemble_the_result(pkg, tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    out = str(tmp_path / "y.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    y = np.load(out)
    a = wl.overlap_uniform(n=400, kappa=1e3)
    ref = oracle.invroot(a.rowptr, a.colind, a.vals, 2)
    assert np.array_equal(y, ref)


def test_more_shards_than_rows_tile_with_empty_shards(pkg):
    a = wl.overlap_small(n=5)
    ranges = [pkg.shard_rows(a.rowptr, 8, k) for k in range(8)]
    assert ranges[0][0] == 0 and ranges[-1][1] == a.n
    for (b0, e0), (b1, e1) in zip(ranges, ranges[1:]):
        assert e0 == b1 and b0 <= e0
    assert sum(e - b for b, e in ranges) == a.n
    assert any(e == b for b, e in ranges)          # some shards hold no row
