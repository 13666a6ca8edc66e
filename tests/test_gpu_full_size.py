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
