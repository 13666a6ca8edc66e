"""Tensor-core (tcgen05) modes vs the FP64 oracle through the C ABI.

OZAKI (exact-slice BF16) must match within 1e-7 Ha absolute, the mixed-path
tolerance.  BF16x3 and TF32x3 accumulate in the tensor cores' FP32 and are
held to their measured accuracy class (relative 1e-5 of E(T)); single-pass
TF32 to 1e-3 relative."""
import numpy as np
import pytest

import tegen
from oracle import t_energy as O
from gpu_common import check_inputs_match, golden, need_gpu, shuffled

pytestmark = pytest.mark.gpu

MODES = ["ozaki", "bf16x3", "tf32x3"]


def tol(prec, ref):
    if prec == "ozaki":
        return 1e-7
    if prec == "tf32":
        return 1e-3 * abs(ref)
    return 1e-5 * abs(ref) + 1e-9


@pytest.fixture(scope="module")
def te():
    return need_gpu()


@pytest.mark.parametrize("prec", MODES)
def test_small_first_case(te, prec):
    cl = tegen.make_cluster(3, 17, 80, 4)
    ref = float(O.t_energy(O.inputs(**cl.arrays())))
    h = te.Handle(0)
    e = float(te.t_energy(cl, prec, handle=h))
    h.sync()
    assert abs(e - ref) <= tol(prec, ref), (e, ref)


@pytest.mark.parametrize("prec", MODES)
def test_o8v40_total_and_shares(te, prec):
    g = golden("o8v40")
    cl = tegen.make_cluster(*tegen.WORKLOADS["o8v40"])
    check_inputs_match(cl, g)
    e = float(te.t_energy(cl, prec))
    assert abs(e - g["e_t"]) <= min(1e-7, tol(prec, g["e_t"]))
    sh = te.t_energy_triples(cl, precision=prec).cpu().numpy()
    ref = np.array(g["shares"])
    atol = 1e-10 if prec == "ozaki" else 1e-8
    np.testing.assert_allclose(sh, ref, rtol=0, atol=atol)


def test_tf32_single_pass_is_close(te):
    g = golden("o8v40")
    cl = tegen.make_cluster(*tegen.WORKLOADS["o8v40"])
    e = float(te.t_energy(cl, "tf32"))
    assert abs(e - g["e_t"]) <= tol("tf32", g["e_t"])


@pytest.mark.parametrize("prec", MODES)
@pytest.mark.parametrize("o,v,seed", [(2, 3, 1), (3, 7, 2), (2, 9, 3), (5, 11, 5), (4, 33, 6),
                                      (6, 65, 7), (3, 130, 8), (2, 200, 9), (3, 260, 10)])
def test_ragged_shapes_unsorted_eps(te, prec, o, v, seed):
    cl = tegen.make_cluster(o, v, 4 * (o + v), seed)
    arrs = shuffled(cl.arrays(), seed)
    arrs["t1"] = arrs["t1"] * 100.0
    ref = float(O.t_energy(O.inputs(**arrs)))
    e = float(te.t_energy(arrs, prec))
    assert abs(e - ref) <= tol(prec, ref), (e, ref)


@pytest.mark.parametrize("prec", MODES)
def test_deterministic_and_homogeneous(te, prec):
    cl = tegen.make_cluster(4, 24, 96, 2)
    a = cl.arrays()
    e0 = te.t_energy(a, prec).item()
    assert te.t_energy(a, prec).item() == e0
    s = dict(a, **{n: a[n] * 2.0 for n in ("ovvv", "ooov", "ovov", "t1", "t2")})
    assert te.t_energy(s, prec).item() == 16.0 * e0


@pytest.mark.parametrize("prec", MODES)
def test_o16v120_matches_golden(te, prec):
    g = golden("o16v120")
    cl = tegen.make_cluster(*tegen.WORKLOADS["o16v120"])
    check_inputs_match(cl, g)
    e = float(te.t_energy(cl, prec))
    assert abs(e - g["e_t"]) <= tol(prec, g["e_t"]), (e, g["e_t"])
    if prec == "ozaki":
        sh = te.t_energy_triples(cl, precision=prec).cpu().numpy()
        np.testing.assert_allclose(sh, np.array(g["shares"]), rtol=0, atol=1e-9)
