"""Fragment-projected E(T) (t_energy_frag) through the C ABI, float64 ("fp64")
and exact-slice ("ozaki"):

* totals and per-triple shares against the oracle's projected energy, on
  ragged shapes with unsorted orbital energies, for a fragment projector and
  for a general (non-symmetric) matrix;
* the identity projector gives t_energy's value;
* projectors of a partition of the occupied space add up to t_energy;
* nocc=16 nvir=120: sampled per-triple shares against stored oracle values
  (tests/golden/oracle_o16v120_frag.json), and exact-slice against float64;
* determinism and argument checks."""
import numpy as np
import pytest
import torch

import tegen
from oracle import t_energy as O
from gpu_common import check_inputs_match, golden, need_gpu, shuffled

pytestmark = pytest.mark.gpu

NAMES = ("eps_o", "eps_v", "ovvv", "ooov", "ovov", "t1", "t2")
ETOL = {"fp64": 1e-10, "ozaki": 1e-7}  # Ha, absolute
RTOL = {"fp64": 1e-11, "ozaki": 1e-6}  # and relative to the energy


@pytest.fixture(scope="module")
def te():
    return need_gpu()


def dev(arrs):
    return {n: torch.as_tensor(np.ascontiguousarray(arrs[n])).cuda() for n in NAMES}


def projector(o, nf, seed):
    u, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((o, o)))
    return u[:, :nf] @ u[:, :nf].T


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
@pytest.mark.parametrize("o,v,seed", [(2, 3, 1), (3, 7, 2), (4, 12, 3), (5, 17, 4), (3, 40, 5), (2, 70, 6)])
def test_matches_oracle(te, o, v, seed, prec):
    arrs = shuffled(tegen.make_cluster(o, v, 4 * (o + v), seed).arrays(), seed)
    arrs["t1"] = arrs["t1"] * 50.0
    c = O.inputs(**arrs)
    blocks = O._blocks(c)
    rng = np.random.default_rng(seed)
    for cf in (projector(o, max(1, o // 2), seed), rng.standard_normal((o, o))):
        ref = float(O.t_energy_projected(c, cf))
        e, sh = te.t_energy_frag(dev(arrs), cf, prec, shares=True)
        assert abs(float(e) - ref) <= ETOL[prec] and abs(float(e) - ref) <= RTOL[prec] * abs(ref) + 1e-16, \
            (float(e), ref)
        ref_sh = [float(O.triple_share_projected(c, cf, *t, blocks)) for t in O.unique_triples(o)]
        sh = sh.cpu().numpy()
        scale = max(abs(x) for x in ref_sh) if ref_sh else 1.0
        for t, (a, b) in enumerate(zip(sh, ref_sh)):
            assert abs(a - b) <= RTOL[prec] * scale, (t, a, b)


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_identity_is_the_cluster_energy(te, prec):
    """C^f = I gives t_energy's E(T): to 1e-12 relative in float64; in exact
    slices both sit within 1e-8 relative of the float64 energy (the projected
    energy's strided GEMMs scale each slab or pair block on its own, the
    contraction kernel one scale per array, so their last bits differ)."""
    a = dev(tegen.make_cluster(*tegen.WORKLOADS["o8v40"]).arrays())
    e = float(te.t_energy(a, prec))
    ef = float(te.t_energy_frag(a, np.eye(8), prec))
    if prec == "fp64":
        assert abs(ef - e) <= 1e-12 * abs(e)
    else:
        e64 = float(te.t_energy(a, "fp64"))
        assert abs(ef - e64) <= 1e-8 * abs(e64) and abs(e - e64) <= 1e-8 * abs(e64), (ef, e, e64)


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_partition_of_unity(te, prec):
    o = 8
    a = dev(tegen.make_cluster(*tegen.WORKLOADS["o8v40"]).arrays())
    u, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((o, o)))
    total = 0.0
    for cols in (slice(0, 3), slice(3, 5), slice(5, 8)):
        f = u[:, cols]
        total += float(te.t_energy_frag(a, f @ f.T, prec))
    e = float(te.t_energy(a, "fp64"))
    assert abs(total - e) <= (1e-11 if prec == "fp64" else 1e-7) * abs(e) + (0 if prec == "fp64" else 1e-7)


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_o16v120_sampled_shares_vs_golden(te, prec):
    """float64: 1e-12 relative per share; exact-slice: 1e-9 Ha per share (the
    per-share bar of the unprojected energy at this size)."""
    g = golden("o16v120_frag")
    cl = tegen.make_cluster(g["nocc"], g["nvir"], g["naux"], g["seed"])
    check_inputs_match(cl, g)
    _, sh = te.t_energy_frag(dev(cl.arrays()), np.array(g["cf"]), prec, shares=True)
    sh = sh.cpu().numpy()
    for idx, ref in zip(g["triple_index"], g["shares"]):
        tol = 1e-12 * abs(ref) + 1e-18 if prec == "fp64" else 1e-9
        assert abs(sh[idx] - ref) <= tol, (idx, sh[idx], ref)


def test_exact_slice_against_float64_o16v120(te):
    a = dev(tegen.make_cluster(*tegen.WORKLOADS["o16v120"]).arrays())
    cf = projector(16, 6, 16)
    e64, s64 = te.t_energy_frag(a, cf, "fp64", shares=True)
    eoz, soz = te.t_energy_frag(a, cf, "ozaki", shares=True)
    assert abs(float(eoz) - float(e64)) <= 1e-7
    assert float((soz - s64).abs().max()) <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_deterministic(te, prec):
    a = dev(tegen.make_cluster(4, 24, 112, 2).arrays())
    cf = projector(4, 2, 1)
    e0, s0 = te.t_energy_frag(a, cf, prec, shares=True)
    e1, s1 = te.t_energy_frag(a, cf, prec, shares=True)
    assert float(e0) == float(e1) and torch.equal(s0, s1)


def test_single_occupied_orbital_gives_zero(te):
    a = dev(tegen.make_cluster(1, 9, 40, 3).arrays())
    assert float(te.t_energy_frag(a, np.eye(1), "fp64")) == 0.0


def test_arguments_are_checked(te):
    a = dev(tegen.make_cluster(3, 10, 52, 1).arrays())
    with pytest.raises(te.TEnergyError):
        te.t_energy_frag(a, np.eye(3), "bf16x3")
    with pytest.raises(ValueError):
        te.t_energy_frag(a, np.eye(4), "fp64")
