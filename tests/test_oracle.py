"""Pins of the FP64 oracle against things other than itself.

* an independent spin-orbital formulation of (T) (``spin_orbital_ref``);
* exact invariants of the formula: E = 0 for one occupied orbital, additivity
  over non-interacting clusters, relabelling invariance, power-of-two
  homogeneity, affinity in t1, Euler identities of the gradient;
* central finite differences of the energy for the gradient;
* planted mistakes in the oracle (dropped factor, wrong sign, transposed
  operand, wrong weight) that the spin-orbital pin must catch.
"""
import itertools

import numpy as np
import pytest
import torch

import tegen
from oracle import t_energy as O
from spin_orbital_ref import spin_orbital_t_energy

TINY = [(2, 3, 12, 5), (3, 4, 20, 1), (3, 5, 16, 2), (4, 3, 10, 9)]


def _cluster(o, v, naux, seed, t1_scale=1.0, shuffle=False):
    cl = tegen.make_cluster(o, v, naux, seed)
    eri = tegen.eri_full(o, v, naux, seed)
    arrs = cl.arrays()
    arrs["t1"] = arrs["t1"] * t1_scale
    if shuffle:  # unsorted orbital energies: relabel occupied and virtual orbitals
        rng = np.random.default_rng(seed + 100)
        po = rng.permutation(o)
        pv = rng.permutation(v)
        arrs = _relabel(arrs, po, pv)
        perm = np.concatenate([po, o + pv])
        eri = eri[np.ix_(perm, perm, perm, perm)]
    return arrs, eri


def _relabel(a, po, pv):
    return dict(
        eps_o=a["eps_o"][po], eps_v=a["eps_v"][pv],
        ovvv=a["ovvv"][np.ix_(po, pv, pv, pv)],
        ooov=a["ooov"][np.ix_(po, po, po, pv)],
        ovov=a["ovov"][np.ix_(po, pv, po, pv)],
        t1=a["t1"][np.ix_(po, pv)],
        t2=a["t2"][np.ix_(po, po, pv, pv)])


def _spin(arrs, eri, o):
    return spin_orbital_t_energy(eri, o, arrs["eps_o"], arrs["eps_v"], arrs["t1"], arrs["t2"])


@pytest.mark.parametrize("o,v,naux,seed", TINY)
@pytest.mark.parametrize("t1_scale,shuffle", [(1.0, False), (300.0, True)])
def test_matches_spin_orbital_form(o, v, naux, seed, t1_scale, shuffle):
    arrs, eri = _cluster(o, v, naux, seed, t1_scale, shuffle)
    e_or = float(O.t_energy(O.inputs(**arrs)))
    e_so = _spin(arrs, eri, o)
    assert e_so != 0.0
    assert abs(e_or - e_so) <= 1e-12 * abs(e_so)


@pytest.mark.parametrize("o,v,naux,seed", TINY[:3])
def test_three_forms_agree(o, v, naux, seed):
    arrs, _ = _cluster(o, v, naux, seed, 300.0)
    c = O.inputs(**arrs)
    e_u = float(O.t_energy(c))
    e_o = float(O.t_energy_ordered(c))
    e_r = float(O.t_energy_restricted(c))
    assert abs(e_u - e_o) <= 1e-13 * abs(e_o)
    assert abs(e_r - e_o) <= 1e-13 * abs(e_o)


def test_random_nonsymmetric_inputs_forms_agree():
    # no symmetry of ints or amplitudes: the forms must still agree
    rng = np.random.default_rng(4)
    o, v = 3, 4
    arrs = dict(eps_o=-1 - rng.random(o), eps_v=1 + rng.random(v),
                ovvv=rng.standard_normal((o, v, v, v)), ooov=rng.standard_normal((o, o, o, v)),
                ovov=rng.standard_normal((o, v, o, v)), t1=rng.standard_normal((o, v)),
                t2=rng.standard_normal((o, o, v, v)))
    c = O.inputs(**arrs)
    e_u = float(O.t_energy(c))
    e_r = float(O.t_energy_restricted(c))
    e_o = float(O.t_energy_ordered(c))
    assert abs(e_u - e_r) <= 1e-12 * abs(e_r)
    assert abs(e_o - e_r) <= 1e-12 * abs(e_r)


def test_one_occupied_orbital_is_exactly_zero():
    arrs, _ = _cluster(1, 6, 20, 3, 300.0)
    c = O.inputs(**arrs)
    assert float(O.t_energy_restricted(c)) == 0.0
    assert float(O.t_energy(c)) == 0.0
    assert float(O.triple_energy(c, 0, 0, 0)) == 0.0


def _direct_sum(a, b):
    oa, va = a["t1"].shape
    ob, vb = b["t1"].shape
    o, v = oa + ob, va + vb
    out = dict(eps_o=np.concatenate([a["eps_o"], b["eps_o"]]),
               eps_v=np.concatenate([a["eps_v"], b["eps_v"]]),
               ovvv=np.zeros((o, v, v, v)), ooov=np.zeros((o, o, o, v)),
               ovov=np.zeros((o, v, o, v)), t1=np.zeros((o, v)), t2=np.zeros((o, o, v, v)))
    A = (slice(0, oa), slice(0, va))
    B = (slice(oa, o), slice(va, v))
    for (so, sv), src in ((A, a), (B, b)):
        out["ovvv"][so, sv, sv, sv] = src["ovvv"]
        out["ooov"][so, so, so, sv] = src["ooov"]
        out["ovov"][so, sv, so, sv] = src["ovov"]
        out["t1"][so, sv] = src["t1"]
        out["t2"][so, so, sv, sv] = src["t2"]
    return out


def test_additive_over_noninteracting_clusters():
    a, _ = _cluster(2, 4, 12, 11, 300.0)
    b, _ = _cluster(3, 3, 14, 12, 300.0)
    ea = float(O.t_energy(O.inputs(**a)))
    eb = float(O.t_energy(O.inputs(**b)))
    eab = float(O.t_energy(O.inputs(**_direct_sum(a, b))))
    assert abs(eab - (ea + eb)) <= 1e-13 * (abs(ea) + abs(eb))


def test_relabelling_invariance():
    arrs, _ = _cluster(3, 5, 16, 2, 300.0)
    e0 = float(O.t_energy(O.inputs(**arrs)))
    rng = np.random.default_rng(0)
    for _ in range(2):
        e1 = float(O.t_energy(O.inputs(**_relabel(arrs, rng.permutation(3), rng.permutation(5)))))
        assert abs(e1 - e0) <= 1e-13 * abs(e0)


def test_power_of_two_homogeneity_is_exact():
    arrs, _ = _cluster(3, 4, 20, 1, 300.0)
    e0 = float(O.t_energy(O.inputs(**arrs)))
    scaled = dict(arrs)
    for n in ("ovvv", "ooov", "ovov", "t1", "t2"):
        scaled[n] = arrs[n] * 2.0
    assert float(O.t_energy(O.inputs(**scaled))) == 16.0 * e0
    eps = dict(arrs, eps_o=arrs["eps_o"] * 4.0, eps_v=arrs["eps_v"] * 4.0)
    assert float(O.t_energy(O.inputs(**eps))) == e0 / 4.0


def test_affine_in_t1():
    arrs, _ = _cluster(3, 4, 20, 1, 300.0)
    e = lambda s: float(O.t_energy(O.inputs(**dict(arrs, t1=arrs["t1"] * s))))
    e0, e1, e2 = e(0.0), e(1.0), e(2.0)
    assert abs(e2 - 2 * e1 + e0) <= 1e-13 * abs(e2)
    assert abs(e1 - e0) > 1e-6 * abs(e1)   # the t1 term is not negligible here


def test_gradient_matches_central_differences():
    arrs, _ = _cluster(2, 3, 12, 5, 300.0)
    c = O.inputs(**arrs)
    e, g = O.t_energy_grad(c)
    rng = np.random.default_rng(1)
    h = 1e-5
    for name in O.NAMES:
        x = arrs[name]
        flat_idx = rng.choice(x.size, size=min(6, x.size), replace=False)
        for fi in flat_idx:
            idx = np.unravel_index(fi, x.shape)
            xp = x.copy(); xp[idx] += h
            xm = x.copy(); xm[idx] -= h
            ep = float(O.t_energy(O.inputs(**dict(arrs, **{name: xp}))))
            em = float(O.t_energy(O.inputs(**dict(arrs, **{name: xm}))))
            fd = (ep - em) / (2 * h)
            an = float(g[name][idx])
            scale = max(float(g[name].abs().max()), 1e-300)
            assert abs(fd - an) <= 1e-6 * scale, (name, idx, fd, an)


def test_gradient_euler_identities():
    arrs, _ = _cluster(3, 4, 20, 1, 300.0)
    c = O.inputs(**arrs)
    e, g = O.t_energy_grad(c)
    deg4 = sum(float((torch.from_numpy(arrs[n]) * g[n]).sum())
               for n in ("ovvv", "ooov", "ovov", "t1", "t2"))
    degm1 = sum(float((torch.from_numpy(arrs[n]) * g[n]).sum()) for n in ("eps_o", "eps_v"))
    assert abs(deg4 - 4 * e) <= 1e-12 * abs(e)
    assert abs(degm1 + e) <= 1e-12 * abs(e)


# --- planted mistakes: each must break the spin-orbital pin ---------------

def _mut_drop_half(c, i, j, k, orig=O.y_disconnected):
    return 2.0 * orig(c, i, j, k)


def _mut_sign_ooov(c, p, q, r):
    return (torch.einsum("abd,cd->abc", c.ovvv[p], c.t2[r, q])
            + torch.einsum("la,lbc->abc", c.ooov[q, :, p, :], c.t2[:, r]))


def _mut_transposed_t2(c, p, q, r):
    return (torch.einsum("abd,cd->abc", c.ovvv[p], c.t2[q, r])
            - torch.einsum("la,lbc->abc", c.ooov[q, :, p, :], c.t2[:, r]))


def _mut_r_cycle(x):
    i, j, k = x.ijk
    return ((4.0 * x(i, j, k) - 2.0 * x(k, j, i) - 2.0 * x(i, k, j))
            + (x(k, i, j) + x(j, k, i) - 2.0 * x(j, k, i)))


def _mut_weight(i, j, k):
    return 6


MUTATIONS = [("y_disconnected", _mut_drop_half), ("x_bracket", _mut_sign_ooov),
             ("x_bracket", _mut_transposed_t2), ("r_operator", _mut_r_cycle),
             ("triple_multiplicity", _mut_weight)]


@pytest.mark.parametrize("name,fn", MUTATIONS, ids=[m[1].__name__ for m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, fn):
    arrs, eri = _cluster(3, 4, 20, 1, 300.0)
    e_so = _spin(arrs, eri, 3)
    monkeypatch.setattr(O, name, fn)
    e_bad = float(O.t_energy(O.inputs(**arrs)))
    assert abs(e_bad - e_so) > 1e-9 * abs(e_so)
