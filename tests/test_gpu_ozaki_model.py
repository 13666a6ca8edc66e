"""The exact-slice tensor-core mode against a float64 model of its own
arithmetic (numpy, written here from the slicing scheme, independent of the
library): every array is scaled by a power of two from its largest magnitude
(all four K segments share one unit), cut into four 7-bit slices by repeated
round-to-nearest, and the slice products with i + j <= 3 are kept.

The two agree to ~1e-11 relative per triple, far below the scheme's own error
(~1e-7 relative against exact float64): this pins the claims that the
level-2 and level-3 accumulators are exact and that the hi/lo G pairs and the
double-float epilogue add nothing measurable."""
import math

import numpy as np
import pytest
import torch

import tegen
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    return need_gpu()


def _slices(x, s, n=4, beta=7):
    t = x * 2.0 ** (-s)
    out = []
    for k in range(n):
        t = t * 2.0 ** beta
        m = np.rint(t)
        t = t - m
        out.append(m * 2.0 ** (s - beta * (k + 1)))
    return out


def _kept(SA, SB, maxlev):
    return [(SA[i], sum(SB[j] for j in range(len(SB)) if i + j <= maxlev)) for i in range(len(SA))
            if i <= maxlev]


def model_share(a, i, j, k, nslices=4, beta=7):
    """float64 model of the exact-slice arithmetic: slice products a_i b_j
    with i + j <= nslices - 1 kept."""
    maxlev = nslices - 1
    eo, ev, ovvv, ooov, ovov, t1, t2 = (a[n] for n in ("eps_o", "eps_v", "ovvv", "ooov", "ovov", "t1", "t2"))
    ex = lambda x: math.frexp(float(np.max(np.abs(x))))[1]
    Eovvv, Et2, Eooov = ex(ovvv), ex(t2), ex(ooov)
    U = max(Eovvv + Et2, Et2 + Eooov)
    sl = lambda x, e: _slices(x, e, nslices, beta)
    s1 = _kept(sl(ovvv, U - Et2), sl(t2, Et2), maxlev)
    s3 = _kept(sl(t2, U - Eooov), sl(ooov, Eooov), maxlev)

    def G(p, q, r):
        g = 0.0
        for A, B in s1:
            g = g + np.einsum("xyd,zd->xyz", A[p], B[r, q], optimize=True) + np.einsum("yxd,zd->xyz", A[q], B[r, p], optimize=True)
        for A, B in s3:
            g = g - np.einsum("lyx,lz->xyz", A[:, p], B[q, :, r], optimize=True) - np.einsum("lxy,lz->xyz", A[:, q], B[p, :, r], optimize=True)
        return g

    W = G(i, j, k) + G(j, k, i).transpose(2, 0, 1) + G(k, i, j).transpose(1, 2, 0)
    ovs = 0.5 * (ovov + ovov.transpose(2, 3, 0, 1))
    Y = (np.einsum("ab,c->abc", ovs[i, :, j, :], t1[k]) + np.einsum("bc,a->abc", ovs[j, :, k, :], t1[i])
         + np.einsum("ac,b->abc", ovs[i, :, k, :], t1[j]))
    V = W + Y
    RV = (4 * V + V.transpose(1, 2, 0) + V.transpose(2, 0, 1)
          - 2 * (V.transpose(2, 1, 0) + V.transpose(0, 2, 1) + V.transpose(1, 0, 2)))
    D = eo[i] + eo[j] + eo[k] - ev[:, None, None] - ev[None, :, None] - ev[None, None, :]
    m = 3 if (i == j or j == k) else 6
    return m / 3.0 * float(np.sum(W * RV / D))


def canonical(o):
    return [(i, j, k) for i in range(o) for j in range(i + 1) for k in range(j + 1) if not (i == j == k)]


@pytest.mark.parametrize("bits,nslices,rtol,scheme_min", [(7, 4, 1e-9, 1e-9), (6, 5, 1e-9, 1e-11)])
def test_matches_slice_model_o16v120(te, bits, nslices, rtol, scheme_min):
    cl = tegen.make_cluster(*tegen.WORKLOADS["o16v120"])
    arrs = cl.arrays()
    a = {n: torch.as_tensor(np.ascontiguousarray(x)).cuda() for n, x in arrs.items()}
    tri = canonical(16)
    h = te.Handle(0)
    h.set_ozaki_bits(bits)
    sh = te.t_energy_triples(a, precision="ozaki", handle=h).cpu().numpy()
    ref64 = te.t_energy_triples(a, precision="fp64", handle=h).cpu().numpy()
    picks = list(np.argsort(np.abs(ref64))[-4:]) + [0, 137, 401]
    # the approximate higher-level accumulator and the float32 Y carry errors
    # relative to the largest products, hence the absolute floor
    floor = 1e-12 * float(np.max(np.abs(ref64)))
    worst_scheme = 0.0
    for t in picks:
        m = model_share(arrs, *tri[t], nslices=nslices, beta=bits)
        print(bits, t, tri[t], sh[t] - m, m - ref64[t], ref64[t])
        assert abs(sh[t] - m) <= rtol * abs(m) + floor, (t, tri[t], sh[t], m)
        worst_scheme = max(worst_scheme, abs(m - ref64[t]) / abs(ref64[t]))
    # the model is not the float64 value: the comparison above is not vacuous
    assert worst_scheme > scheme_min


def test_six_bit_slices_beyond_k1024(te):
    """2 (nvir + nocc) = 1034 > 1024: the automatic choice is 6-bit slicing;
    7-bit slicing is refused; the result meets the mixed-mode bar against the
    float64 path (itself held to the oracle at 1e-10 on the ragged shapes)."""
    from paper_2412_18553_gb300._lib import TE_EUNSUPPORTED
    cl = tegen.make_cluster(2, 515, 2068, 21)
    a = {n: torch.as_tensor(np.ascontiguousarray(x)).cuda() for n, x in cl.arrays().items()}
    h = te.Handle(0)
    e64 = float(te.t_energy(a, "fp64", handle=h))
    e6 = float(te.t_energy(a, "ozaki", handle=h))
    assert abs(e6 - e64) <= 1e-7, (e6, e64)
    h.set_ozaki_bits(7)
    with pytest.raises(te.TEnergyError) as ei:
        te.t_energy(a, "ozaki", handle=h)
    assert ei.value.status == TE_EUNSUPPORTED
    h.set_ozaki_bits(6)
    assert float(te.t_energy(a, "ozaki", handle=h)) == e6
