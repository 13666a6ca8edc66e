"""The o32v320 workload at full size, in the launch configuration the bench
times: the float64 path on single-triple ranges and the exact-slice tensor-core
path over the whole cluster (t_energy_triples over all triples runs the same
batches as t_energy), compared on the triples whose oracle shares are stored
in tests/golden/oracle_o32v320_sample.json (written by make_golden.py from the
oracle alone).

The exact-slice mode's per-triple error is that of its slicing scheme (the
dropped slice products of order 2^-28 relative to the largest products; up to
~2e-8 Ha on the largest shares here, reproduced by a float64 model of the
scheme in test_gpu_ozaki_model.py), so each share is held to the 1e-7 Ha bar
that E(T) itself must meet."""
import numpy as np
import pytest
import torch

import tegen
from gpu_common import check_inputs_match, golden, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    return need_gpu()


@pytest.fixture(scope="module")
def case():
    g = golden("o32v320_sample")
    cl = tegen.make_cluster(g["nocc"], g["nvir"], g["naux"], g["seed"])
    check_inputs_match(cl, g)
    arrs = {n: torch.as_tensor(np.ascontiguousarray(x)).cuda() for n, x in cl.arrays().items()}
    return g, arrs


def test_fp64_sampled_triples(te, case):
    g, a = case
    for t, ref in zip(g["triple_index"], g["shares"]):
        sh = float(te.t_energy_triples(a, t, t + 1, precision="fp64")[0])
        assert abs(sh - ref) <= 1e-12 * max(1.0, abs(ref)), (t, sh, ref)


def test_ozaki_whole_cluster_sampled_and_summed(te, case):
    g, a = case
    h = te.Handle(0)
    n = te.num_unique_triples(g["nocc"])
    sh = te.t_energy_triples(a, 0, n, precision="ozaki", handle=h)
    e = float(te.t_energy(a, "ozaki", handle=h))
    h.sync()
    s = sh.cpu().numpy()
    for t, ref in zip(g["triple_index"], g["shares"]):
        assert abs(s[t] - ref) <= 1e-7, (t, s[t], ref)
    assert abs(float(np.sum(s)) - e) <= 1e-10 * abs(e)


class _OvvvRows:
    """The rows ovvv[p] the oracle reads for one triple, copied from the
    device tensor the GPU path uses (the full array is 67 GB)."""

    def __init__(self, dev_ovvv, rows):
        self._rows = {p: dev_ovvv[p].double().cpu() for p in set(rows)}

    def __getitem__(self, p):
        return self._rows[int(p)]


def test_o48v560_sampled_triples():
    """nocc=48 nvir=560 (seed 7): K = 2 (v + o) = 1216 > 1024, so the
    exact-slice mode runs with 6-bit slices.  ovvv is formed on the GPU by
    the generator; the oracle reads the same values (row copies) for two
    triples: the largest share (47,47,46) and a distinct-index triple."""
    from oracle import t_energy as O
    te = need_gpu()
    o, v, naux, seed = tegen.WORKLOADS["o48v560"]
    cl = tegen.make_cluster(o, v, naux, seed, device="cuda")
    torch.cuda.empty_cache()
    arrs = cl.arrays()
    a = {n: (x if isinstance(x, torch.Tensor) else torch.as_tensor(np.ascontiguousarray(x)).cuda())
         for n, x in arrs.items()}
    tri = [(i, j, k) for i in range(o) for j in range(i + 1) for k in range(j + 1) if not (i == j == k)]
    h = te.Handle(0)
    for (i, j, k) in [(47, 47, 46), (40, 25, 3)]:
        t = tri.index((i, j, k))
        small = O.inputs(arrs["eps_o"], arrs["eps_v"], np.zeros((1, 1, 1, 1)), arrs["ooov"], arrs["ovov"],
                         arrs["t1"], arrs["t2"])
        small.ovvv = _OvvvRows(a["ovvv"], (i, j, k))
        ref = float(O.triple_share(small, i, j, k))
        e64 = float(te.t_energy_triples(a, t, t + 1, precision="fp64", handle=h)[0])
        eoz = float(te.t_energy_triples(a, t, t + 1, precision="ozaki", handle=h)[0])
        h.sync()
        assert abs(e64 - ref) <= 1e-12 * max(1.0, abs(ref)), ((i, j, k), e64, ref)
        assert abs(eoz - ref) <= 1e-7, ((i, j, k), eoz, ref)


def test_o24v240_whole_cluster_exact_slice_within_1e7_of_float64():
    """nocc=24 nvir=240 (seed 2): E(T) of the whole cluster in the exact-slice
    mode against the float64 GPU path, |dE| <= 1e-7 Ha (the accuracy bar of
    the mixed path) on the total rather than per share.  The float64 path is
    held to the oracle on two triples of the same cluster: the heaviest and
    one with distinct indices."""
    from oracle import t_energy as O
    te = need_gpu()
    o, v, naux, seed = tegen.WORKLOADS["o24v240"]
    cl = tegen.make_cluster(o, v, naux, seed)
    a = {n: torch.as_tensor(np.ascontiguousarray(x)).cuda() for n, x in cl.arrays().items()}
    h = te.Handle(0)
    e64 = float(te.t_energy(a, "fp64", handle=h))
    eoz = float(te.t_energy(a, "ozaki", handle=h))
    h.sync()
    assert abs(eoz - e64) <= 1e-7, (eoz, e64)
    c = O.inputs(**cl.arrays())
    trip = O.unique_triples(o)
    for ijk in [(23, 23, 22), (17, 9, 2)]:
        t = trip.index(ijk)
        ref = float(O.triple_share(c, *ijk))
        got = float(te.t_energy_triples(a, t, t + 1, precision="fp64", handle=h)[0])
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (ijk, got, ref)
    h.sync()


def test_o48v560_adjoint_on_a_sampled_triple():
    """nocc=48 nvir=560 (seed 7): the adjoint of one canonical triple
    (t_energy_vjp_triples) with exact-slice contractions against the float64
    adjoint of the same triple, at each input's 64 largest float64 entries
    and 64 seeded ones, within 1e-6 of the input's largest float64 magnitude;
    and the float64 adjoint against central differences (step 1e-5) of the
    float64 share at each input's two largest entries.  Gradients are asked
    for in two groups (ovvv alone, then the rest) to keep the device's memory
    within bounds: ovvv and its gradient are 67 GB each."""
    te = need_gpu()
    torch.cuda.empty_cache()
    names = ("eps_o", "eps_v", "ovvv", "ooov", "ovov", "t1", "t2")
    o, v, naux, seed = tegen.WORKLOADS["o48v560"]
    cl = tegen.make_cluster(o, v, naux, seed, device="cuda")
    a = {n: (x if isinstance(x, torch.Tensor) else torch.as_tensor(np.ascontiguousarray(x)).cuda())
         for n, x in cl.arrays().items()}
    del cl
    torch.cuda.empty_cache()
    tri = [(i, j, k) for i in range(o) for j in range(i + 1) for k in range(j + 1) if not (i == j == k)]
    t = tri.index((40, 25, 3))
    h = te.Handle(0)
    gen = torch.Generator(device="cuda").manual_seed(3)
    samples = {}

    def pick(n, g):
        # the 64 largest entries (within the three nonzero rows of d ovvv: a
        # row has v^3 = 1.8e8 entries, while the whole tensor's 8.4e9 exceed
        # what a single torch.topk handles) and 64 seeded entries
        if n == "ovvv":
            rows = sorted({40, 25, 3})
            cand = torch.cat([g[p].reshape(-1).abs().topk(64).indices + p * g[p].numel() for p in rows])
            top = cand[g.view(-1)[cand].abs().argsort(descending=True)[:64]]
            mx = max(float(g[p].abs().max()) for p in rows)
        else:
            flat = g.view(-1)
            top = flat.abs().topk(min(64, flat.numel())).indices
            mx = float(flat.abs().max())
        idx = torch.cat([top, torch.randint(0, g.numel(), (64,), device="cuda", generator=gen)])
        return idx, g.view(-1)[idx].clone(), mx

    for grp in (("ovvv",), tuple(n for n in names if n != "ovvv")):
        e64, g64 = te.t_energy_vjp_triples(a, t, t + 1, precision="fp64", handle=h, grads=grp)
        for n in grp:
            samples[n] = pick(n, g64[n])
        del g64
        torch.cuda.empty_cache()
        eoz, goz = te.t_energy_vjp_triples(a, t, t + 1, precision="ozaki", handle=h, grads=grp)
        for n in grp:
            idx, ref, mx = samples[n]
            err = float((goz[n].view(-1)[idx] - ref).abs().max())
            assert err <= 1e-6 * mx, (n, err, mx)
        del goz
        torch.cuda.empty_cache()
    h.sync()
    assert abs(float(eoz) - float(e64)) <= 1e-7, (float(eoz), float(e64))
    step = 1e-5
    for n in names:
        idx, ref, mx = samples[n]
        flat = a[n].view(-1)
        for q in range(2):
            i = idx[q:q + 1]
            keep = flat[i].clone()
            flat[i] = keep + step
            ep = float(te.t_energy_triples(a, t, t + 1, precision="fp64", handle=h)[0])
            flat[i] = keep - step
            em = float(te.t_energy_triples(a, t, t + 1, precision="fp64", handle=h)[0])
            flat[i] = keep
            fd = (ep - em) / (2 * step)
            assert abs(fd - float(ref[q])) <= 1e-6 * mx, (n, q, fd, float(ref[q]), mx)
    h.sync()
