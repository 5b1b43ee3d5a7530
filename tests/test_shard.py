"""Root-range sharding across ranks: two gloo ranks on CPU, the oracle standing in
for each rank's GPU count of its root range."""
import os
import socket

import numpy as np
import pytest

import bipgen
import oracle


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_root_ranges_cover_and_balance():
    from paper_2403_07858_gb300.shard import root_ranges
    w = np.array([1, 1, 1, 10, 1, 1, 1, 1, 1, 1], dtype=float)
    for world in (1, 2, 3, 4, 16):
        rs = root_ranges(w, world)
        assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == len(w)
        assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
    rs = root_ranges(np.ones(1000), 4)
    assert [b - a for a, b in rs] == [250, 250, 250, 250]
    assert root_ranges([], 3) == [(0, 0)] * 3


def _worker(rank, world, port, p, q, anchor, result_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2403_07858_gb300.shard import allreduce_u128, root_ranges
    g = bipgen.workload_small()
    deg = np.diff(g.off_u if anchor == "U" else g.off_v).astype(float)
    r0, r1 = root_ranges(deg ** 2, world)[rank]
    mine = oracle.count(g, p, q, anchor=anchor, roots=(r0, r1))
    total = allreduce_u128(mine)
    big = allreduce_u128((1 << 126) + rank * (3 << 95))  # limbs carry across ranks
    try:
        allreduce_u128((1 << 127) + rank)  # 2^128 + 1 in total
        overflow = 0
    except OverflowError:
        overflow = 1
    if rank == 0:
        with open(result_path, "w") as f:
            f.write(f"{total} {big} {overflow}")
    dist.destroy_process_group()


@pytest.mark.parametrize("p,q,anchor", [(3, 3, "U"), (4, 3, "V")])
def test_two_gloo_ranks_sum_to_the_whole_count(tmp_path, p, q, anchor):
    import torch.multiprocessing as tmp_mp
    out = tmp_path / "res.txt"
    tmp_mp.start_processes(_worker, args=(2, _free_port(), p, q, anchor, str(out)), nprocs=2,
                           start_method="spawn")
    total, big, overflow = map(int, out.read_text().split())
    assert total == oracle.count(bipgen.workload_small(), p, q)
    assert big == 2 * (1 << 126) + (3 << 95)
    assert overflow == 1
