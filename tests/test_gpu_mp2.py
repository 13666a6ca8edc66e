"""The MP2 step (t_mp2_bno_batched) through the C ABI against the oracle
(oracle/mp2.py): amplitudes, both 1-RDM blocks and the BNO populations, in
float64 and with the contractions in exact BF16 slices.

Tolerances, relative to each output's largest magnitude: float64 1e-13
(amplitudes, densities) and 1e-12 (populations, from the Jacobi solver);
exact slices 1e-7: the (ia|jb) contraction carries 28 bits of the DF factor
relative to its largest entry (measured: amplitudes within 5e-9, densities
and populations within 2e-8 of their largest entry, up to nocc=20 nvir=200);
the density contractions are float64 in both modes.  Particle number tr gamma_oo + tr gamma_vv = 2 nocc and symmetry
hold on the GPU's own output; the v = 8 nocc batch's two smallest members
run in one call with a larger one."""
import numpy as np
import pytest
import torch

import tegen
from oracle import mp2 as M
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-13, "ozaki": 1e-7}
POP_TOL = {"fp64": 1e-12, "ozaki": 1e-7}


@pytest.fixture(scope="module")
def te():
    return need_gpu()


def check(out, ref, prec):
    for n in ("t2", "gamma_oo", "gamma_vv"):
        a, b = out[n].cpu().numpy(), ref[n]
        scale = max(np.abs(b).max(), 1e-300)
        assert np.abs(a - b).max() <= TOL[prec] * scale, (n, np.abs(a - b).max(), scale)
    for n in ("pop_o", "pop_v"):
        a, b = out[n].cpu().numpy(), ref[n]
        scale = max(np.abs(b).max(), 1e-300)
        assert np.all(np.diff(a) >= 0.0), n
        assert np.abs(a - b).max() <= POP_TOL[prec] * scale, (n, np.abs(a - b).max(), scale)
    o = out["gamma_oo"].shape[0]
    goo, gvv = out["gamma_oo"].cpu().numpy(), out["gamma_vv"].cpu().numpy()
    assert abs(np.trace(goo) + np.trace(gvv) - 2 * o) <= (1e-12 if prec == "fp64" else 1e-7) * o
    assert np.abs(goo - goo.T).max() <= TOL[prec] * 2.0
    assert np.abs(gvv - gvv.T).max() <= TOL[prec] * max(np.abs(gvv).max(), 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
@pytest.mark.parametrize("o,v,naux,seed", [(1, 5, 12, 1), (2, 3, 10, 2), (3, 7, 30, 3), (4, 16, 80, 4),
                                           (5, 33, 150, 5), (7, 61, 272, 6)])
def test_matches_oracle(te, prec, o, v, naux, seed):
    c = tegen.mp2_inputs(o, v, naux, seed)
    out = te.mp2_bno_batched([c], prec)[0]
    check(out, M.mp2_bno(*c), prec)


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_batch_members(te, prec):
    """Members 11 and 14 of the v = 8 nocc batch (nocc 9, nvir 72) and member
    6 (nocc 13, nvir 104) in one call, each against the oracle."""
    cs = tegen.mp2_batch([11, 6, 14], rule="v8o")
    outs = te.mp2_bno_batched(cs, prec)
    for c, out in zip(cs, outs):
        check(out, M.mp2_bno(*c), prec)


def test_amplitudes_are_the_cluster_t2(te):
    """The float64 amplitudes are the t2 input of the (T) energy for the same
    draw (the generator forms t2 from the same integrals on the host)."""
    o, v, naux, seed = tegen.WORKLOADS["o8v40"]
    cl = tegen.make_cluster(o, v, naux, seed)
    c = tegen.mp2_inputs(o, v, naux, seed)
    out = te.mp2_bno_batched([c], "fp64", outputs=("t2",))[0]
    np.testing.assert_allclose(out["t2"].cpu().numpy(), cl.t2, rtol=0, atol=1e-15 * np.abs(cl.t2).max())


def test_exact_slices_vs_float64_at_a_larger_size(te):
    """nocc=20 nvir=200 naux=880: the two modes agree (oracle-free: the float64
    path is held to the oracle above)."""
    c = tegen.mp2_inputs(20, 200, 880, 9)
    a, b = te.mp2_bno_batched([c], "fp64")[0], te.mp2_bno_batched([c], "ozaki")[0]
    for n in ("t2", "gamma_oo", "gamma_vv", "pop_o", "pop_v"):
        x, y = a[n].cpu().numpy(), b[n].cpu().numpy()
        assert np.abs(x - y).max() <= 1e-7 * np.abs(x).max(), n


def test_checks(te):
    c = list(tegen.mp2_inputs(3, 9, 40, 7))
    h = te.Handle(0)
    bad = c[2].copy()
    bad[1, 1, 2] = np.nan
    te.mp2_bno_batched([c, (c[0], c[1], bad)], "fp64", handle=h)
    with pytest.raises(te.TEnergyError) as ei:
        h.sync()
    assert ei.value.status == 1 and "Bov" in str(ei.value) and "cluster 1" in str(ei.value)
    with pytest.raises(te.TEnergyError):
        te.mp2_bno_batched([c], "bf16x3", handle=h)
    with pytest.raises(te.TEnergyError):
        te.mp2_bno_batched([c], "fp64", outputs=(), handle=h)
    h.sync()
