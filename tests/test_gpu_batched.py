"""t_energy_batched: many independent clusters (Eq. C_f: E = sum_x E_x) in one
captured CUDA graph, checked against single-cluster calls and the oracle."""
import numpy as np
import pytest
import torch

import tegen
from oracle import t_energy as O
from gpu_common import need_gpu, shuffled

pytestmark = pytest.mark.gpu

SIZES = [(3, 17, 4), (5, 24, 5), (2, 9, 6), (6, 40, 7), (4, 33, 8), (1, 12, 9), (7, 57, 10)]


def _batch():
    out = []
    for o, v, seed in SIZES:
        cl = tegen.make_cluster(o, v, 4 * (o + v), seed)
        a = shuffled(cl.arrays(), seed)
        a["t1"] = a["t1"] * 30.0
        out.append(a)
    return out


@pytest.fixture(scope="module")
def te():
    return need_gpu()


@pytest.fixture(scope="module")
def batch():
    return _batch()


@pytest.fixture(scope="module")
def ref(batch):
    return [float(O.t_energy(O.inputs(**a))) for a in batch]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("ozaki", 1e-7)])
def test_batched_matches_oracle_and_single_calls(te, batch, ref, prec, tol):
    h = te.Handle(0)
    dev = [{n: torch.as_tensor(x).cuda() for n, x in a.items()} for a in batch]
    eb = te.t_energy_batched(dev, prec, handle=h).cpu().numpy()
    for x, a in enumerate(dev):
        assert abs(eb[x] - ref[x]) <= tol, (x, eb[x], ref[x])
        single = te.t_energy(a, prec, handle=h).item()
        assert single == eb[x]
    # a second call replays the captured graph: bitwise the same
    eb2 = te.t_energy_batched(dev, prec, handle=h).cpu().numpy()
    assert np.array_equal(eb, eb2)
    h.sync()


def test_batched_graph_sees_new_data(te, batch):
    h = te.Handle(0)
    dev = [{n: torch.as_tensor(x).cuda() for n, x in a.items()} for a in batch[:3]]
    e1 = te.t_energy_batched(dev, "fp64", handle=h).cpu().numpy()
    for a in dev:  # scale amplitudes in place: E scales by 4 (E is quadratic in t)
        a["t2"].mul_(2.0)
        a["t1"].mul_(2.0)
    e2 = te.t_energy_batched(dev, "fp64", handle=h).cpu().numpy()
    np.testing.assert_array_equal(e2, 4.0 * e1)


def test_batched_v8o_sixteen_ozaki(te):
    clusters = tegen.make_batch(range(16), rule="v8o")
    h = te.Handle(0)
    dev = [{n: torch.as_tensor(x).cuda() for n, x in c.arrays().items()} for c in clusters]
    eb = te.t_energy_batched(dev, "ozaki", handle=h).cpu().numpy()
    # sampled members against the FP64 path
    for x in (0, 7, 15):
        e64 = te.t_energy(dev[x], "fp64", handle=h).item()
        assert abs(eb[x] - e64) <= 1e-7, (x, eb[x], e64)


def test_uneven_batch_members_sampled(te):
    """Members of the 96-cluster uneven batch (seeds 0..95: nocc ~ [10,40],
    nvir ~ nocc U[8,12]), the smallest and the median one, run batched in the
    exact-slice mode.  Batched totals equal single-cluster calls bit for bit;
    the smallest member's total meets the bar against the float64 path; two
    triples of each member match the oracle (float64 path 1e-12 relative,
    exact-slice mode 1e-7 Ha)."""
    order = sorted(range(96), key=lambda s: tegen.batch_sizes(s)[0] * tegen.batch_sizes(s)[1] ** 3)
    picks = [order[0], order[48]]
    clusters = tegen.make_batch(picks, rule="uneven")
    h = te.Handle(0)
    dev = [{n: torch.as_tensor(x).cuda() for n, x in c.arrays().items()} for c in clusters]
    eb = te.t_energy_batched(dev, "ozaki", handle=h).cpu().numpy()
    for x, c in enumerate(clusters):
        assert te.t_energy(dev[x], "ozaki", handle=h).item() == eb[x]
        if x == 0:
            e64 = te.t_energy(dev[x], "fp64", handle=h).item()
            assert abs(eb[x] - e64) <= 1e-7, (picks[x], eb[x], e64)
        inp = O.inputs(**c.arrays())
        tri = O.unique_triples(c.nocc)
        for t in (0, len(tri) - 1):
            ref = float(O.triple_share(inp, *tri[t]))
            got = te.t_energy_triples(dev[x], t, t + 1, precision="fp64", handle=h).item()
            assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (picks[x], t, got, ref)
            got = te.t_energy_triples(dev[x], t, t + 1, precision="ozaki", handle=h).item()
            assert abs(got - ref) <= 1e-7, (picks[x], t, got, ref)
    h.sync()
