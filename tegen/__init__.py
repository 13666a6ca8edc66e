"""Seeded synthetic closed-shell clusters for the (T) energy.

This module produces the inputs that both the CUDA path and the FP64 oracle
consume.  It holds none of the (T) arithmetic: it draws orbital energies and a
density-fitting factor, forms the integral blocks and the MP2-style t2.

Recipe (one cluster, ``make_cluster(nocc, nvir, naux, seed)``), drawn from
``numpy.random.default_rng(seed)`` in this order:

1. ``eps_o`` = sorted U[-1.5, -0.4] Ha, ``nocc`` values;
2. ``eps_v`` = sorted U[0.2, 4.0] Ha, ``nvir`` values;
3. ``B[P,p,q]`` = N(0,1) * 0.05 * exp(-|p-q|/10) over n = nocc+nvir orbitals
   (occupied first), then symmetrised ``B <- (B + B^T)/2`` in (p,q);
4. ``t1`` = N(0,1) * 1e-3, shape [nocc, nvir].

Integrals are chemists' notation ``(pq|rs) = sum_P B[P,p,q] B[P,r,s]``:

* ``ovvv[i,a,b,d] = (ia|bd)``   shape [o][v][v][v]
* ``ooov[j,l,i,a] = (jl|ia)``   shape [o][o][o][v]
* ``ovov[i,a,j,b] = (ia|jb)``   shape [o][v][o][v]
* ``t2[i,j,a,b] = (ia|jb) / (e_i + e_j - e_a - e_b)`` shape [o][o][v][v]

Everything is formed in FP64 on the host, except ``ovvv`` for large clusters
(``2*o*v^3*naux`` above ``HOST_FLOP_LIMIT``), which ``device="cuda"`` forms
with a library GEMM on the GPU in split-BF16 (three products, FP32
accumulation) and stores as FP64; forming it in FP64 would cost more than the
(T) energy itself.  The arrays produced are the inputs: every consumer reads the
same FP64 values.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

HOST_FLOP_LIMIT = 2.0e13

__all__ = [
    "Cluster",
    "make_cluster",
    "batch_sizes",
    "make_batch",
    "mp2_inputs",
    "mp2_batch",
    "WORKLOADS",
    "eri_full",
]


@dataclass
class Cluster:
    nocc: int
    nvir: int
    eps_o: np.ndarray
    eps_v: np.ndarray
    ovvv: object  # numpy array, or torch tensor on the GPU for large clusters
    ooov: np.ndarray
    ovov: np.ndarray
    t1: np.ndarray
    t2: np.ndarray
    meta: dict = field(default_factory=dict)
    Bov: object = None  # [naux][o][v] density-fitting factor blocks (with_df=True)
    Bvv: object = None  # [naux][v][v]

    def arrays(self):
        return dict(eps_o=self.eps_o, eps_v=self.eps_v, ovvv=self.ovvv,
                    ooov=self.ooov, ovov=self.ovov, t1=self.t1, t2=self.t2)


def _draw(nocc, nvir, naux, rng):
    n = nocc + nvir
    eps_o = np.sort(rng.uniform(-1.5, -0.4, nocc))
    eps_v = np.sort(rng.uniform(0.2, 4.0, nvir))
    idx = np.arange(n)
    env = 0.05 * np.exp(-np.abs(idx[:, None] - idx[None, :]) / 10.0)
    B = rng.standard_normal((naux, n, n)) * env[None]
    B = 0.5 * (B + B.transpose(0, 2, 1))
    t1 = rng.standard_normal((nocc, nvir)) * 1e-3
    return eps_o, eps_v, B, t1


def _ovvv_host(Bov, Bvv):
    naux, o, v = Bov.shape
    lhs = Bov.reshape(naux, o * v).T          # [(i,a), P]
    rhs = Bvv.reshape(naux, v * v)            # [P, (b,d)]
    return (lhs @ rhs).reshape(o, v, v, v)


def _ovvv_cuda(Bov, Bvv):
    import torch
    naux, o, v = Bov.shape
    dev = torch.device("cuda")
    lhs = torch.from_numpy(np.ascontiguousarray(Bov.reshape(naux, o * v).T)).to(dev)
    rhs = torch.from_numpy(np.ascontiguousarray(Bvv.reshape(naux, v * v))).to(dev)

    def split(x):
        # x = hi + lo + O(2^-16 |x|); both parts are BF16 values held in FP32,
        # so a TF32 GEMM multiplies them exactly and accumulates in FP32
        hi = x.to(torch.bfloat16)
        lo = (x - hi.to(torch.float64)).to(torch.bfloat16)
        return hi.to(torch.float32), lo.to(torch.float32)

    lh, ll = split(lhs)
    rh, rl = split(rhs)
    del lhs, rhs
    out = torch.empty((o * v, v * v), dtype=torch.float64, device=dev)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        step = max(256, (1 << 28) // max(1, o * v))
        for c0 in range(0, v * v, step):
            c1 = min(v * v, c0 + step)
            acc = torch.matmul(lh, rh[:, c0:c1])
            acc += torch.matmul(lh, rl[:, c0:c1])
            acc += torch.matmul(ll, rh[:, c0:c1])
            out[:, c0:c1] = acc.to(torch.float64)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out.reshape(o, v, v, v)


def make_cluster(nocc: int, nvir: int, naux: int, seed: int, device: str = "cpu",
                 rng=None, host_flop_limit: float = HOST_FLOP_LIMIT, with_df: bool = False,
                 form_ovvv: bool = True) -> Cluster:
    """Draw one synthetic cluster.  ``device="cuda"`` forms ovvv on the GPU
    (returned as a CUDA float64 tensor) when it costs more than
    ``host_flop_limit`` flops; smaller ones are formed on the host in FP64 and
    returned as numpy arrays.  ``with_df`` attaches the factor blocks Bov
    [naux][o][v] and Bvv [naux][v][v] (numpy, C-contiguous); ``form_ovvv=False``
    leaves ovvv as None (the factors then stand for it)."""
    if rng is None:
        rng = np.random.default_rng(seed)
    eps_o, eps_v, B, t1 = _draw(nocc, nvir, naux, rng)
    o, v = nocc, nvir
    Boo = np.ascontiguousarray(B[:, :o, :o])
    Bov = np.ascontiguousarray(B[:, :o, o:])
    Bvv = np.ascontiguousarray(B[:, o:, o:])
    ovov = (Bov.reshape(naux, o * v).T @ Bov.reshape(naux, o * v)).reshape(o, v, o, v)
    ooov = (Boo.reshape(naux, o * o).T @ Bov.reshape(naux, o * v)).reshape(o, o, o, v)
    d2 = (eps_o[:, None, None, None] + eps_o[None, :, None, None]
          - eps_v[None, None, :, None] - eps_v[None, None, None, :])
    t2 = ovov.transpose(0, 2, 1, 3) / d2
    flops = 2.0 * o * v ** 3 * naux
    if not form_ovvv:
        ovvv, how = None, "not formed"
    elif device == "cuda" and flops > host_flop_limit:
        ovvv = _ovvv_cuda(Bov, Bvv)
        how = "gpu-split-bf16x3"
    else:
        ovvv = _ovvv_host(Bov, Bvv)
        how = "host-fp64"
    return Cluster(o, v, eps_o, eps_v, ovvv, ooov, ovov, t1,
                   np.ascontiguousarray(t2),
                   meta=dict(naux=naux, seed=seed, ovvv_formed=how),
                   Bov=Bov if with_df else None, Bvv=Bvv if with_df else None)


def mp2_inputs(nocc: int, nvir: int, naux: int, seed: int, rng=None):
    """The MP2 step's inputs for the same draw as ``make_cluster``: (eps_o,
    eps_v, Bov) with Bov[P, i, a] the occupied-virtual block of the
    density-fitting factor, C-contiguous float64."""
    if rng is None:
        rng = np.random.default_rng(seed)
    eps_o, eps_v, B, _ = _draw(nocc, nvir, naux, rng)
    return eps_o, eps_v, np.ascontiguousarray(B[:, :nocc, nocc:])


def mp2_batch(seeds, rule="v8o"):
    """MP2 inputs of batch members (sizes as in ``make_batch``)."""
    out = []
    for s in seeds:
        o, v, naux, rng = batch_sizes(s, rule)
        out.append(mp2_inputs(o, v, naux, s, rng=rng))
    return out


def eri_full(nocc: int, nvir: int, naux: int, seed: int) -> np.ndarray:
    """Full (pq|rs) over all n orbitals for the same draw (tiny clusters only)."""
    rng = np.random.default_rng(seed)
    _, _, B, _ = _draw(nocc, nvir, naux, rng)
    n = nocc + nvir
    Bf = B.reshape(naux, n * n)
    return (Bf.T @ Bf).reshape(n, n, n, n)


def batch_sizes(seed: int, rule: str = "uneven"):
    """Cluster sizes of a batch member.  ``"uneven"``: nocc ~ integers[10,40],
    nvir = round-half-even(nocc * U[8,12]), naux = 4(nocc+nvir).  ``"v8o"``:
    nocc ~ integers[8,20], nvir = 8 nocc, naux = 4(nocc+nvir).  The sizes are
    the first draws of ``default_rng(seed)``; the cluster continues from the
    same generator."""
    rng = np.random.default_rng(seed)
    if rule == "uneven":
        o = int(rng.integers(10, 41))
        v = int(np.round(o * rng.uniform(8.0, 12.0)))
    elif rule == "v8o":
        o = int(rng.integers(8, 21))
        v = 8 * o
    else:
        raise ValueError(rule)
    return o, v, 4 * (o + v), rng


def make_batch(seeds, rule="uneven", device="cpu", host_flop_limit=HOST_FLOP_LIMIT):
    out = []
    for s in seeds:
        o, v, naux, rng = batch_sizes(s, rule)
        out.append(make_cluster(o, v, naux, s, device=device, rng=rng, host_flop_limit=host_flop_limit))
    return out


# Named single-cluster workloads: (nocc, nvir, naux, seed).
WORKLOADS = {
    "o8v40": (8, 40, 160, 0),
    "o32v320": (32, 320, 1280, 1),
    "o16v120": (16, 120, 544, 3),
    "o48v560": (48, 560, 2432, 7),
    # between the two: whole-cluster comparison of the exact-slice and float64 paths
    "o24v240": (24, 240, 960, 2),
    # same virtual space as o32v320 with 8 occupied orbitals: kernel profiling
    # at full tile shapes with a few GB on the device
    "o8v320": (8, 320, 1280, 1),
}
