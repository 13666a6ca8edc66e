"""Sharding of E(T) across ranks (host logic only).

Clusters do not interact (Eq. C_f), and the energy of one cluster is a sum of
independent per-triple shares, so the path shards with one scalar exchange:

* independent clusters: ``assign_clusters`` spreads a batch over ranks by
  longest-processing-time first on the flop count;
* one cluster: rank r evaluates the contiguous canonical triple range
  ``triple_range(nocc, r, world)`` with ``t_energy_triples``; E is the sum of
  the per-rank partial sums, gathered and added in rank order so the result
  does not depend on the reduction tree of the backend.
"""
from __future__ import annotations

import heapq

import torch

from . import num_unique_triples


def triple_range(nocc: int, rank: int, world: int):
    """[t0, t1) of canonical unique triples for ``rank``: contiguous, sizes
    differing by at most one, covering every triple exactly once."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of size {world}")
    n = num_unique_triples(nocc)
    base, extra = divmod(n, world)
    t0 = rank * base + min(rank, extra)
    return t0, t0 + base + (1 if rank < extra else 0)


def assign_clusters(flops, world: int):
    """Longest-processing-time-first assignment: clusters sorted by decreasing
    flop count (ties by index) go to the least-loaded rank (ties by rank).
    Returns one list of cluster indices per rank, each in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(flops)), key=lambda x: (-float(flops[x]), x))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for x in order:
        load, r = heapq.heappop(heap)
        out[r].append(x)
        heapq.heappush(heap, (load + float(flops[x]), r))
    return [sorted(v) for v in out]


def sharded_energy(cluster, precision: str = "ozaki", group=None, handle=None, shares_fn=None) -> float:
    """E(T) of one cluster split over the ranks of ``group`` (default: the
    world).  ``shares_fn(cluster, t0, t1)`` returns the per-triple shares of
    the range (default: the library's ``t_energy_triples``).  Every rank
    returns the same value."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    eps_o = cluster["eps_o"] if isinstance(cluster, dict) else cluster.eps_o
    nocc = int(eps_o.shape[0])
    t0, t1 = triple_range(nocc, rank, world)
    if shares_fn is None:
        from . import t_energy_triples
        shares_fn = lambda c, a, b: t_energy_triples(c, a, b, precision=precision, handle=handle)
    part = torch.zeros((1,), dtype=torch.float64)
    if t1 > t0:
        sh = torch.as_tensor(shares_fn(cluster, t0, t1)).to("cpu", torch.float64)
        part[0] = float(sh.sum())
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else None
    if dev is not None:
        part = part.to(dev)
    parts = [torch.zeros_like(part) for _ in range(world)]
    dist.all_gather(parts, part, group=group)
    total = 0.0
    for p in parts:  # rank order
        total += float(p.item())
    return total
