"""Host logic of the multi-rank paths on the CPU (gloo, world size 2): the
triple-range split covers every triple once, the cluster assignment is a
deterministic longest-first balance, and the sharded sum over two ranks of
oracle shares equals the oracle's E(T)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import tegen
from oracle import t_energy as O
from paper_2412_18553_gb300 import num_unique_triples
from paper_2412_18553_gb300.shard import assign_clusters, sharded_energy, triple_range


@pytest.mark.parametrize("nocc", [1, 2, 3, 5, 8, 17])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_triple_ranges_partition(nocc, world):
    n = num_unique_triples(nocc)
    got = []
    sizes = []
    for r in range(world):
        t0, t1 = triple_range(nocc, r, world)
        got.extend(range(t0, t1))
        sizes.append(t1 - t0)
    assert got == list(range(n))
    assert max(sizes) - min(sizes) <= 1


def test_assign_clusters_balances_and_is_deterministic():
    flops = [5, 1, 9, 3, 3, 7, 2, 8]
    a = assign_clusters(flops, 3)
    assert a == assign_clusters(list(flops), 3)
    assert sorted(x for part in a for x in part) == list(range(len(flops)))
    loads = [sum(flops[x] for x in part) for part in a]
    assert max(loads) - min(loads) <= max(flops)
    assert assign_clusters(flops, 1) == [list(range(len(flops)))]


def _shares(c, t0, t1):
    inp = O.inputs(**c)
    tri = O.unique_triples(inp.nocc)[t0:t1]
    return torch.tensor([float(O.triple_share(inp, *t)) for t in tri], dtype=torch.float64)


def _worker(rank, world, port, arrs, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = sharded_energy(arrs, shares_fn=_shares)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_sum_two_ranks_gloo():
    arrs = tegen.make_cluster(4, 10, 56, 5).arrays()
    ref = float(O.t_energy(O.inputs(**arrs)))
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), arrs, out), nprocs=2, join=True,
                           start_method="spawn")
        vals = [out[0], out[1]]
    assert vals[0] == vals[1]
    assert abs(vals[0] - ref) <= 1e-14 * abs(ref) + 1e-18
