"""Multi-rank host logic on CPU (gloo, world size 2): the block-row partition of a triangle
over ranks (disjoint, covering, balanced slices of the packed output) and the max-over-ranks
timing reduction the benchmark uses."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1308_1419_gb300.build import build_libtd  # noqa: E402

build_libtd()
from paper_1308_1419_gb300 import td  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, cases, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for N, rho in cases:
            mine = torch.tensor(td.td_partition(N, rho, world, rank), dtype=torch.int64)
            got = [torch.zeros(4, dtype=torch.int64) for _ in range(world)]
            dist.all_gather(got, mine)
            if rank == 0:
                q.put(((N, rho), [g.tolist() for g in got]))
        # the benchmark's step time is the maximum over ranks
        t = torch.tensor([10.0 + rank])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            q.put(("max", float(t.item())))
    finally:
        dist.destroy_process_group()


def test_partition_over_two_gloo_ranks():
    cases = [(65536, 16), (1000, 8), (7, 32), (16384, 128)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_worker, args=(2, _free_port(), cases, q), nprocs=2, join=True, start_method="spawn")
    results = dict(q.get() for _ in range(len(cases) + 1))
    assert results["max"] == 11.0
    for N, rho in cases:
        parts = results[(N, rho)]
        total = N * (N + 1) // 2
        nb = -(-N // rho)
        assert parts[0][0] == 0 and parts[-1][1] == nb and parts[0][2] == 0 and parts[-1][3] == total
        for a, b in zip(parts, parts[1:]):
            assert a[1] == b[0] and a[3] == b[2]          # contiguous, disjoint
        if N >= 64 * rho:
            sizes = [p[3] - p[2] for p in parts]
            assert max(sizes) - min(sizes) <= 2 * rho * N  # balanced to within a block row


def test_partition_many_ranks_single_process():
    for N, rho, G in [(65536, 16, 8), (30720, 16, 3), (100, 8, 16)]:
        parts = [td.td_partition(N, rho, G, r) for r in range(G)]
        assert parts[0][2] == 0 and parts[-1][3] == N * (N + 1) // 2
        for a, b in zip(parts, parts[1:]):
            assert a[1] == b[0] and a[3] == b[2]
    with pytest.raises(td.TDError):
        td.td_partition(100, 8, 2, 2)
