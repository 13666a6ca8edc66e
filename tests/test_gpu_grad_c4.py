"""The adjoint at the gradient workload, through the C ABI, in float64 and in
exact BF16 slices:

* nocc=16 nvir=120 naux=544 (seed 3): sampled gradient entries (64 per input
  plus each input's largest entry) against the oracle's reverse-mode
  gradient stored in tests/golden/oracle_o16v120_grad.json (written by
  make_golden.py from the oracle alone), relative to each input's largest
  gradient magnitude: 1e-6 (the bar for gradients) in the exact-slice mode,
  1e-10 in float64;
* central differences with step 1e-5 of the float64 energy at the largest
  sampled entries of every input, and along one direction per input spread
  over all its sampled entries;
* the 16-cluster batch (seeds 0..15, nocc 8..20, nvir = 8 nocc) in one
  t_energy_vjp_batched call: its two smallest members against their stored
  oracle gradient samples, and members against single t_energy_vjp calls
  (bit for bit: the same code runs per member)."""
import json
import os

import numpy as np
import pytest
import torch

import tegen
from gpu_common import HERE, check_inputs_match, need_gpu

pytestmark = pytest.mark.gpu

NAMES = ("eps_o", "eps_v", "ovvv", "ooov", "ovov", "t1", "t2")
RTOL = {"fp64": 1e-10, "ozaki": 1e-6}
STEP = 1e-5


@pytest.fixture(scope="module")
def te():
    return need_gpu()


def load(name):
    with open(os.path.join(HERE, "golden", f"oracle_{name}_grad.json")) as f:
        return json.load(f)


def dev(arrs):
    return {n: torch.as_tensor(np.ascontiguousarray(arrs[n])).cuda() for n in NAMES}


def check_samples(g, ref, rtol):
    for n in NAMES:
        r = ref["grad"][n]
        got = g[n].reshape(-1)[torch.as_tensor(r["index"], device=g[n].device)].cpu().numpy()
        err = float(np.max(np.abs(got - np.array(r["value"]))))
        assert err <= rtol * r["max_abs"], (n, err, r["max_abs"])
        # the largest magnitude of the whole tensor, a property of every entry
        assert abs(float(g[n].abs().max()) - r["max_abs"]) <= rtol * r["max_abs"], n


@pytest.fixture(scope="module")
def o16v120():
    ref = load("o16v120")
    cl = tegen.make_cluster(ref["nocc"], ref["nvir"], ref["naux"], ref["seed"])
    check_inputs_match(cl, ref)
    return ref, dev(cl.arrays())


@pytest.fixture(scope="module")
def grads(te, o16v120):
    _, a = o16v120
    out = {}
    for prec in ("fp64", "ozaki"):
        e, g = te.t_energy_vjp(a, precision=prec)
        out[prec] = (float(e), g)
    return out


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_o16v120_against_oracle_gradient(te, o16v120, grads, prec):
    ref, _ = o16v120
    e, g = grads[prec]
    assert abs(e - ref["e_t"]) <= (1e-10 if prec == "fp64" else 1e-7)
    check_samples(g, ref, RTOL[prec])


def test_o16v120_central_differences(te, o16v120, grads):
    """dE/dx by (E(x + h) - E(x - h)) / 2h, h = 1e-5, float64 energies: at the
    three largest sampled entries of every input, and along a random-sign
    direction over all its sampled entries.  E is quadratic in any one entry
    of ovvv, ooov and t2 and linear in one of ovov and t1, so the difference
    is exact there up to rounding; in eps it is a rational function."""
    ref, a = o16v120
    h = te.Handle(0)
    rng = np.random.default_rng(7)

    def energy_with(n, idx, delta):
        flat = a[n].view(-1)
        keep = flat[idx].clone()
        flat[idx] += delta
        e = float(te.t_energy(a, "fp64", handle=h))
        flat[idx] = keep
        return e

    for n in NAMES:
        r = ref["grad"][n]
        idx = np.array(r["index"])
        val = np.array(r["value"])
        top = idx[np.argsort(-np.abs(val))[:3]]
        ti = torch.as_tensor(top, device="cuda")
        fd = [(energy_with(n, ti[q:q + 1], STEP) - energy_with(n, ti[q:q + 1], -STEP)) / (2 * STEP)
              for q in range(len(top))]
        sgn = torch.as_tensor(rng.choice([-1.0, 1.0], size=len(idx)), device="cuda", dtype=torch.float64)
        ai = torch.as_tensor(idx, device="cuda")
        fd_dir = (energy_with(n, ai, STEP * sgn) - energy_with(n, ai, -STEP * sgn)) / (2 * STEP)
        for prec in ("fp64", "ozaki"):
            g = grads[prec][1][n].reshape(-1)
            an = g[ti].cpu().numpy()
            err = float(np.max(np.abs(np.array(fd) - an)))
            assert err <= 1e-6 * r["max_abs"], (n, prec, fd, an)
            an_dir = float((g[ai] * sgn).sum())
            assert abs(fd_dir - an_dir) <= 1e-6 * r["max_abs"] * np.sqrt(len(idx)), (n, prec, fd_dir, an_dir)
    h.sync()


@pytest.fixture(scope="module")
def batch16():
    cls = tegen.make_batch(range(16), rule="v8o")
    return [dev(c.arrays()) for c in cls], cls


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_batch16_one_call(te, batch16, prec):
    """The batch in one call.  float64 runs a sub-batch (the two stored
    members and one more) to keep the test short; the exact-slice mode runs
    all sixteen."""
    devs, cls = batch16
    ref = load("v8o")
    members = list(range(16)) if prec == "ozaki" else [11, 6, 14]
    gE = [1.0 - 0.1 * x for x in members]
    h = te.Handle(0)
    e, gs = te.t_energy_vjp_batched([devs[x] for x in members], gE=gE, precision=prec, handle=h)
    h.sync()
    pos = {x: q for q, x in enumerate(members)}
    for m in ref["members"]:
        x = m["seed"]
        check_inputs_match(cls[x], m)
        q = pos[x]
        assert abs(float(e[q]) - m["e_t"]) <= (1e-10 if prec == "fp64" else 1e-7)
        scaled = dict(m, grad={n: dict(r, value=[gE[q] * t for t in r["value"]], max_abs=abs(gE[q]) * r["max_abs"])
                               for n, r in m["grad"].items()})
        check_samples(gs[q], scaled, RTOL[prec])
    # members against single calls: the same arithmetic, bit for bit
    for x in (members[1], members[-1]):
        q = pos[x]
        e1, g1 = te.t_energy_vjp(devs[x], gE=gE[q], precision=prec, handle=h)
        assert float(e1) == float(e[q])
        for n in NAMES:
            assert torch.equal(g1[n], gs[q][n]), (x, n)
    h.sync()
