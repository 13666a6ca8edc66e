"""Adjoint of E(T) (t_energy_vjp) through the C ABI, float64 ("fp64") and
with the contractions on the tensor cores in exact BF16 slices ("ozaki").

* element by element against the oracle's reverse-mode gradient, on ragged
  shapes with unsorted orbital energies and on the o8v40 workload (float64:
  1e-10 of each tensor's largest entry; exact-slice: 1e-6, the bar for
  gradients);
* Euler identities (E is homogeneous of degree 4 in the integrals and
  amplitudes together and of degree -1 in the orbital energies);
* central differences of the float64 GPU energy along a random direction;
* the autograd Function's backward is the same adjoint."""
import numpy as np
import pytest
import torch

import tegen
from oracle import t_energy as O
from gpu_common import need_gpu, shuffled

pytestmark = pytest.mark.gpu

NAMES = ("eps_o", "eps_v", "ovvv", "ooov", "ovov", "t1", "t2")
AMPS = ("ovvv", "ooov", "ovov", "t1", "t2")


@pytest.fixture(scope="module")
def te():
    return need_gpu()


def dev(arrs):
    return {n: torch.as_tensor(np.ascontiguousarray(arrs[n])).cuda() for n in NAMES}


def assert_grads_close(g, ref, rtol=1e-10):
    for n in NAMES:
        a = g[n].cpu().numpy()
        b = ref[n].numpy() if isinstance(ref[n], torch.Tensor) else ref[n]
        scale = max(float(np.max(np.abs(b))), 1e-300)
        err = float(np.max(np.abs(a - b)))
        assert err <= rtol * scale, (n, err, scale)


RTOL = {"fp64": 1e-10, "ozaki": 1e-6}
ETOL = {"fp64": 1e-12, "ozaki": 1e-7}


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
@pytest.mark.parametrize("o,v,seed", [(2, 3, 1), (3, 7, 2), (4, 12, 3), (5, 17, 4), (3, 70, 5), (2, 131, 6), (2, 211, 8)])
def test_matches_oracle_gradient(te, o, v, seed, prec):
    cl = tegen.make_cluster(o, v, 4 * (o + v), seed)
    arrs = shuffled(cl.arrays(), seed)
    arrs["t1"] = arrs["t1"] * 50.0
    e_ref, g_ref = O.t_energy_grad(O.inputs(**arrs))
    e, g = te.t_energy_vjp(dev(arrs), precision=prec)
    assert abs(float(e) - e_ref) <= ETOL[prec] * abs(e_ref) + 1e-15
    assert_grads_close(g, g_ref, RTOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_o8v40_matches_oracle_gradient(te, prec):
    cl = tegen.make_cluster(*tegen.WORKLOADS["o8v40"])
    arrs = cl.arrays()
    e_ref, g_ref = O.t_energy_grad(O.inputs(**arrs))
    e, g = te.t_energy_vjp(dev(arrs), gE=-0.75, precision=prec)
    assert abs(float(e) - e_ref) <= ETOL[prec] * abs(e_ref)
    assert_grads_close(g, {n: -0.75 * g_ref[n] for n in NAMES}, RTOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_single_occupied_orbital_gives_zero(te, prec):
    cl = tegen.make_cluster(1, 9, 40, 3)
    e, g = te.t_energy_vjp(dev(cl.arrays()), precision=prec)
    assert float(e) == 0.0
    for n in NAMES:
        assert float(g[n].abs().max()) == 0.0, n


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("ozaki", 1e-6)])
def test_euler_identities(te, prec, tol):
    cl = tegen.make_cluster(6, 48, 216, 11)
    a = dev(cl.arrays())
    e, g = te.t_energy_vjp(a, precision=prec)
    e = float(e)
    deg4 = sum(float((a[n] * g[n]).sum()) for n in AMPS)
    degm1 = sum(float((a[n] * g[n]).sum()) for n in ("eps_o", "eps_v"))
    assert abs(deg4 - 4.0 * e) <= tol * abs(e)
    assert abs(degm1 + e) <= tol * abs(e)


def test_exact_slice_gradient_against_float64_o16v120(te):
    """The nocc=16 nvir=120 workload: the tensor-core adjoint against the
    float64 adjoint, every tensor within 1e-6 of its largest entry."""
    cl = tegen.make_cluster(*tegen.WORKLOADS["o16v120"])
    a = dev(cl.arrays())
    e64, g64 = te.t_energy_vjp(a, precision="fp64")
    eoz, goz = te.t_energy_vjp(a, precision="ozaki")
    assert abs(float(eoz) - float(e64)) <= 1e-7
    assert_grads_close(goz, {n: g64[n].cpu().numpy() for n in NAMES}, 1e-6)


def test_directional_central_difference(te):
    cl = tegen.make_cluster(6, 48, 216, 12)
    a = dev(cl.arrays())
    _, g = te.t_energy_vjp(a)
    gen = torch.Generator().manual_seed(5)
    d = {n: (torch.randn(a[n].shape, generator=gen, dtype=torch.float64) * a[n].abs().mean().cpu()).cuda()
         for n in NAMES}
    h = 1e-4
    ep = float(te.t_energy({n: a[n] + h * d[n] for n in NAMES}, "fp64"))
    em = float(te.t_energy({n: a[n] - h * d[n] for n in NAMES}, "fp64"))
    fd = (ep - em) / (2 * h)
    an = sum(float((g[n] * d[n]).sum()) for n in NAMES)
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_deterministic(te, prec):
    cl = tegen.make_cluster(4, 24, 96, 2)
    a = dev(cl.arrays())
    e0, g0 = te.t_energy_vjp(a, precision=prec)
    e1, g1 = te.t_energy_vjp(a, precision=prec)
    assert float(e0) == float(e1)
    for n in NAMES:
        assert torch.equal(g0[n], g1[n]), n


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_autograd_function_uses_the_adjoint(te, prec):
    cl = tegen.make_cluster(3, 20, 92, 4)
    a = dev(cl.arrays())
    leaves = [a[n].clone().requires_grad_(True) for n in NAMES]
    E = te.TEnergy.apply(*leaves, prec)
    (2.0 * E).backward()
    _, g = te.t_energy_vjp(a, gE=2.0, precision=prec)
    for n, leaf in zip(NAMES, leaves):
        torch.testing.assert_close(leaf.grad, g[n], rtol=1e-13, atol=0)


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_triple_ranges_partition_the_gradient(te, prec):
    """E is additive over triples: the adjoints of ranges that partition the
    canonical triples add up to the whole cluster's adjoint, and their
    energies to E (t_energy_vjp_triples)."""
    cl = tegen.make_cluster(6, 29, 140, 13)
    a = dev(shuffled(cl.arrays(), 13))
    nt = te.num_unique_triples(6)
    e, g = te.t_energy_vjp(a, gE=0.5, precision=prec)
    cuts = [0, 1, 17, nt - 3, nt]
    tot = {n: torch.zeros_like(g[n]) for n in NAMES}
    esum = 0.0
    for b, c in zip(cuts[:-1], cuts[1:]):
        eb, gb = te.t_energy_vjp_triples(a, b, c, gE=0.5, precision=prec)
        esum += float(eb)
        for n in NAMES:
            tot[n] += gb[n]
    assert abs(esum - float(e)) <= 1e-13 * abs(float(e))
    assert_grads_close(tot, {n: g[n].cpu().numpy() for n in NAMES}, 1e-12)
    # an empty range: zero gradient, zero energy
    e0, g0 = te.t_energy_vjp_triples(a, 5, 5, precision=prec)
    assert float(e0) == 0.0 and all(float(g0[n].abs().max()) == 0.0 for n in NAMES)
    with pytest.raises(te.TEnergyError):
        te.t_energy_vjp_triples(a, 3, nt + 1, precision=prec)
