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


def _kept(SA, SB, maxlev=3):
    return [(SA[i], sum(SB[j] for j in range(len(SB)) if i + j <= maxlev)) for i in range(len(SA))]


def model_share(a, i, j, k, maxlev=3):
    eo, ev, ovvv, ooov, ovov, t1, t2 = (a[n] for n in ("eps_o", "eps_v", "ovvv", "ooov", "ovov", "t1", "t2"))
    ex = lambda x: math.frexp(float(np.max(np.abs(x))))[1]
    Eovvv, Et2, Eooov = ex(ovvv), ex(t2), ex(ooov)
    U = max(Eovvv + Et2, Et2 + Eooov)
    s1 = _kept(_slices(ovvv, U - Et2), _slices(t2, Et2), maxlev)
    s3 = _kept(_slices(t2, U - Eooov), _slices(ooov, Eooov), maxlev)

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


def test_matches_slice_model_o16v120(te):
    cl = tegen.make_cluster(*tegen.WORKLOADS["o16v120"])
    arrs = cl.arrays()
    a = {n: torch.as_tensor(np.ascontiguousarray(x)).cuda() for n, x in arrs.items()}
    tri = canonical(16)
    sh = te.t_energy_triples(a, precision="ozaki").cpu().numpy()
    ref64 = te.t_energy_triples(a, precision="fp64").cpu().numpy()
    picks = list(np.argsort(np.abs(ref64))[-4:]) + [0, 137, 401]
    # the approximate level-4/5 accumulator and the float32 Y carry errors
    # relative to the largest products, hence the absolute floor
    floor = 1e-12 * float(np.max(np.abs(ref64)))
    worst_scheme = 0.0
    for t in picks:
        m = model_share(arrs, *tri[t])
        assert abs(sh[t] - m) <= 1e-9 * abs(m) + floor, (t, tri[t], sh[t], m)
        worst_scheme = max(worst_scheme, abs(m - ref64[t]) / abs(ref64[t]))
    # the model is not the float64 value: the comparison above is not vacuous
    assert worst_scheme > 1e-9
