"""Float64 CUDA path vs the FP64 oracle (tolerance 1e-10 Ha absolute on E,
1e-12 Ha per triple share), through the C ABI."""
import numpy as np
import pytest
import torch

import tegen
from oracle import t_energy as O
from gpu_common import check_inputs_match, golden, need_gpu, shuffled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    return need_gpu()


def test_o8v40_total_and_shares(te):
    g = golden("o8v40")
    cl = tegen.make_cluster(*tegen.WORKLOADS["o8v40"])
    check_inputs_match(cl, g)
    e = float(te.t_energy(cl, "fp64"))
    assert abs(e - g["e_t"]) <= 1e-10
    sh = te.t_energy_triples(cl, precision="fp64").cpu().numpy()
    assert sh.shape == (len(g["shares"]),)
    np.testing.assert_allclose(sh, np.array(g["shares"]), rtol=0, atol=1e-12)


@pytest.mark.parametrize("o,v,seed", [(2, 3, 1), (3, 7, 2), (2, 9, 3), (3, 17, 4), (5, 11, 5),
                                      (4, 33, 6), (6, 65, 7)])
def test_tiny_ragged_shapes_unsorted_eps(te, o, v, seed):
    cl = tegen.make_cluster(o, v, 4 * (o + v), seed)
    arrs = shuffled(cl.arrays(), seed)
    arrs["t1"] = arrs["t1"] * 100.0
    ref = float(O.t_energy(O.inputs(**arrs)))
    e = float(te.t_energy(arrs, "fp64"))
    assert abs(e - ref) <= 1e-10 + 1e-12 * abs(ref)
    sh = te.t_energy_triples(arrs, precision="fp64").cpu().numpy()
    c = O.inputs(**arrs)
    ref_sh = [float(O.triple_share(c, *t)) for t in O.unique_triples(o)]
    np.testing.assert_allclose(sh, ref_sh, rtol=1e-11, atol=1e-15)


def test_one_occupied_orbital_gives_zero(te):
    cl = tegen.make_cluster(1, 9, 40, 3)
    assert float(te.t_energy(cl, "fp64")) == 0.0


def test_bitwise_deterministic_and_ranges(te):
    cl = tegen.make_cluster(5, 40, 180, 9)
    e1 = te.t_energy(cl, "fp64").item()
    e2 = te.t_energy(cl, "fp64").item()
    assert e1 == e2
    full = te.t_energy_triples(cl, precision="fp64").cpu()
    part = torch.cat([te.t_energy_triples(cl, 0, 7, "fp64").cpu(),
                      te.t_energy_triples(cl, 7, te.num_unique_triples(5), "fp64").cpu()])
    assert torch.equal(full, part)


def test_power_of_two_homogeneity_is_exact(te):
    cl = tegen.make_cluster(4, 24, 96, 2)
    a = cl.arrays()
    e0 = te.t_energy(a, "fp64").item()
    s = dict(a, **{n: a[n] * 2.0 for n in ("ovvv", "ooov", "ovov", "t1", "t2")})
    assert te.t_energy(s, "fp64").item() == 16.0 * e0


def test_invalid_orbital_energies_rejected(te):
    cl = tegen.make_cluster(3, 8, 40, 1)
    a = cl.arrays()
    a["eps_o"] = a["eps_o"].copy()
    a["eps_o"][1] = a["eps_v"].min() + 0.1
    h = te.Handle(0)
    te.t_energy(a, "fp64", handle=h)  # checked on the device: reported at sync
    with pytest.raises(te.TEnergyError) as ei:
        h.sync()
    assert ei.value.status == 1


def test_o16v120_matches_golden(te):
    g = golden("o16v120")
    cl = tegen.make_cluster(*tegen.WORKLOADS["o16v120"])
    check_inputs_match(cl, g)
    e = float(te.t_energy(cl, "fp64"))
    assert abs(e - g["e_t"]) <= 1e-10
    sh = te.t_energy_triples(cl, precision="fp64").cpu().numpy()
    np.testing.assert_allclose(sh, np.array(g["shares"]), rtol=0, atol=1e-12)
