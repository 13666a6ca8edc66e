"""E(T) with the (ov|vv) block formed on the device from the density-fitting
factors (t_energy_df, t_energy_df_triples) through the C ABI.

The reference is the oracle's E(T) on the oracle's float64 DF product
(oracle/df.py), at the exact-slice bar of 1e-7 Ha; the other tensor-core
modes are held to their accuracy class.  Against the same mode fed with a
float64 ovvv the result agrees far more closely: the formation (five 7-bit
slices per factor, exact level-0/1 sums) is accurate to naux 2^-34 of the
factors' scales, below the 28 bits the contraction keeps of ovvv; what
differs is an occasional last-slice rounding of an ovvv entry (measured up to
3e-10 of E(T); bound 2e-9).  Cases span
one and several K blocks of the formation (naux up to 2049), ragged nvir, and
at nocc=32 nvir=320 several staging groups of slabs, checked on sampled
triples against the float64 path on an ovvv formed by a float64 GEMM."""
import numpy as np
import pytest
import torch

import tegen
from oracle import df as D
from oracle import t_energy as O
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

TOL_ORACLE = {"ozaki": lambda e: 1e-7, "bf16x3": lambda e: 1e-5 * abs(e) + 1e-9,
              "tf32x3": lambda e: 1e-5 * abs(e) + 1e-9, "tf32": lambda e: 1e-3 * abs(e)}


@pytest.fixture(scope="module")
def te():
    return need_gpu()


def oracle_e(cl):
    a = cl.arrays()
    a["ovvv"] = D.ovvv_from_df(cl.Bov, cl.Bvv)
    return float(O.t_energy(O.inputs(**a)))


@pytest.mark.parametrize("o,v,naux,seed", [(2, 8, 30, 1), (3, 17, 80, 4), (5, 33, 150, 2), (8, 40, 192, 0),
                                           (3, 9, 1100, 3), (2, 12, 2049, 5)])
def test_exact_slices_match_oracle(te, o, v, naux, seed):
    cl = tegen.make_cluster(o, v, naux, seed, with_df=True)
    ref = oracle_e(cl)
    h = te.Handle(0)
    e = float(te.t_energy_df(cl, cl.Bov, cl.Bvv, "ozaki", handle=h))
    e_ovvv = float(te.t_energy(cl, "ozaki", handle=h))
    h.sync()
    assert abs(e - ref) <= 1e-7, (e, ref)
    assert abs(e - e_ovvv) <= 2e-9 * abs(ref) + 1e-14, (e, e_ovvv)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "tf32"])
def test_other_modes(te, prec):
    cl = tegen.make_cluster(5, 33, 150, 2, with_df=True)
    ref = oracle_e(cl)
    h = te.Handle(0)
    e = float(te.t_energy_df(cl, cl.Bov, cl.Bvv, prec, handle=h))
    e_ovvv = float(te.t_energy(cl, prec, handle=h))
    h.sync()
    assert abs(e - ref) <= TOL_ORACLE[prec](ref), (e, ref)
    assert abs(e - e_ovvv) <= 1e-8 * abs(ref), (e, e_ovvv)


def test_shares_and_ranges(te):
    cl = tegen.make_cluster(7, 24, 124, 6, with_df=True)
    h = te.Handle(0)
    nt = te.num_unique_triples(7)
    whole = te.t_energy_df_triples(cl, cl.Bov, cl.Bvv, precision="ozaki", handle=h).cpu().numpy()
    parts = np.concatenate([te.t_energy_df_triples(cl, cl.Bov, cl.Bvv, a, b, "ozaki", handle=h).cpu().numpy()
                            for a, b in ((0, 11), (11, 40), (40, nt))])
    e = float(te.t_energy_df(cl, cl.Bov, cl.Bvv, "ozaki", handle=h))
    ref = te.t_energy_triples(cl, precision="ozaki", handle=h).cpu().numpy()
    h.sync()
    np.testing.assert_array_equal(whole, parts)
    np.testing.assert_allclose(whole, ref, rtol=0, atol=1e-12)
    assert abs(e - whole.sum()) <= 1e-12


def test_ovvv_not_read(te):
    """The cluster's ovvv is neither needed nor read: a NaN-filled one changes
    nothing."""
    cl = tegen.make_cluster(4, 20, 96, 8, with_df=True)
    h = te.Handle(0)
    a = cl.arrays()
    e0 = float(te.t_energy_df(a, cl.Bov, cl.Bvv, "ozaki", handle=h))
    a = dict(a)
    a["ovvv"] = np.full_like(a["ovvv"], np.nan)
    e1 = float(te.t_energy_df(a, cl.Bov, cl.Bvv, "ozaki", handle=h))
    del a["ovvv"]
    e2 = float(te.t_energy_df(a, cl.Bov, cl.Bvv, "ozaki", handle=h))
    h.sync()
    assert e0 == e1 == e2


def test_checks(te):
    cl = tegen.make_cluster(3, 10, 40, 9, with_df=True)
    h = te.Handle(0)
    bad = cl.Bvv.copy()
    bad[3, 2, 1] = np.inf
    te.t_energy_df(cl, cl.Bov, bad, "ozaki", handle=h)
    with pytest.raises(te.TEnergyError) as ei:
        h.sync()
    assert ei.value.status == 1 and "Bvv" in str(ei.value)
    bad = cl.Bov.copy()
    bad[0, 0, 0] = np.nan
    te.t_energy_df(cl, bad, cl.Bvv, "ozaki", handle=h)
    with pytest.raises(te.TEnergyError) as ei:
        h.sync()
    assert "Bov" in str(ei.value)
    with pytest.raises(te.TEnergyError) as ei:
        te.t_energy_df(cl, cl.Bov, cl.Bvv, "fp64", handle=h)
    assert ei.value.status == 5
    with pytest.raises(ValueError):
        te.t_energy_df(cl, cl.Bov[:, :2], cl.Bvv, "ozaki", handle=h)
    h.sync()
    assert h.df_workspace_bytes(3, 10, 40) > 0


def test_o32v320_sampled_triples(te):
    """nocc=32 nvir=320 naux=1280 (seed 1), four staging groups of eight
    slabs: sampled shares against the exact-slice path fed with the float64
    DF product (cuBLAS DGEMM on the device), within 1e-8 of the share
    (last-slice roundings of a few of the 1e9 ovvv entries; measured 1.2e-9),
    and
    against the float64 path on it within 2e-8 Ha (the exact-slice shares'
    own accuracy at this size: up to about 1e-8 Ha per triple, while their
    sum over the 5952 triples stays within 1e-7 Ha)."""
    torch.cuda.empty_cache()
    o, v, naux, seed = tegen.WORKLOADS["o32v320"]
    cl = tegen.make_cluster(o, v, naux, seed, with_df=True, form_ovvv=False)
    bov = torch.from_numpy(cl.Bov).cuda()
    bvv = torch.from_numpy(cl.Bvv).cuda()
    a = {n: torch.as_tensor(np.ascontiguousarray(x)).cuda() for n, x in cl.arrays().items() if x is not None}
    a["ovvv"] = (bov.reshape(naux, o * v).T @ bvv.reshape(naux, v * v)).reshape(o, v, v, v).contiguous()
    h = te.Handle(0)
    nt = te.num_unique_triples(o)
    for t in (0, 1777, 4000, nt - 1):
        s_df = float(te.t_energy_df_triples(a, bov, bvv, t, t + 1, "ozaki", handle=h)[0])
        s_oz = float(te.t_energy_triples(a, t, t + 1, "ozaki", handle=h)[0])
        s_64 = float(te.t_energy_triples(a, t, t + 1, "fp64", handle=h)[0])
        assert abs(s_df - s_oz) <= 1e-8 * abs(s_64) + 1e-14, (t, s_df, s_oz)
        assert abs(s_df - s_64) <= 2e-8, (t, s_df, s_64)
    h.sync()
