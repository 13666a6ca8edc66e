"""Pins of the MP2 / BNO oracle (oracle/mp2.py) against what the mathematics
fixes, independently of its own code:

* the unrelaxed MP2 one-body density in spin orbitals, written here from its
  textbook definition (antisymmetrised amplitudes t_IJ^AB = <IJ||AB> / (e_I +
  e_J - e_A - e_B), D_AB = 1/2 sum_IJC t_IJ^AC t_IJ^BC, D_IJ = delta_IJ -
  1/2 sum_KAB t_IK^AB t_JK^AB), summed over the two spins, equals the
  closed-shell blocks of the supplement's BNO section;
* particle number: tr gamma_oo + tr gamma_vv = 2 nocc exactly;
* symmetry of both blocks, invariance of the populations under relabelling
  the occupied or virtual orbitals, the uncorrelated limit (t = 0: gamma_oo =
  2, gamma_vv = 0), and the population sums (trace) and products (det);
* planted mistakes (the exchange sign, the factor 2 of the virtual block, the
  amplitude sign) each break one of these."""
import itertools

import numpy as np
import pytest

import tegen
from oracle import mp2 as M


def draw(o, v, naux, seed):
    eps_o, eps_v, Bov = tegen.mp2_inputs(o, v, naux, seed)
    return eps_o, eps_v, Bov


def spin_orbital_density(eps_o, eps_v, ovov):
    """Spin-summed unrelaxed MP2 density from spin-orbital amplitudes; spin
    orbital 2p + s holds spatial orbital p with spin s."""
    o, v = len(eps_o), len(eps_v)
    no, nv = 2 * o, 2 * v
    T = np.zeros((no, no, nv, nv))
    for I, J, A, B in itertools.product(range(no), range(no), range(nv), range(nv)):
        i, si = divmod(I, 2)
        j, sj = divmod(J, 2)
        a, sa = divmod(A, 2)
        b, sb = divmod(B, 2)
        direct = ovov[i, a, j, b] if (si == sa and sj == sb) else 0.0   # <ij|ab> = (ia|jb)
        exch = ovov[i, b, j, a] if (si == sb and sj == sa) else 0.0     # <ij|ba>
        T[I, J, A, B] = (direct - exch) / (eps_o[i] + eps_o[j] - eps_v[a] - eps_v[b])
    Dvv = 0.5 * np.einsum("ijac,ijbc->ab", T, T)
    Doo = np.eye(no) - 0.5 * np.einsum("ikab,jkab->ij", T, T)
    return Doo[0::2, 0::2] + Doo[1::2, 1::2], Dvv[0::2, 0::2] + Dvv[1::2, 1::2]


@pytest.mark.parametrize("o,v,naux,seed", [(2, 3, 10, 1), (3, 5, 20, 2), (4, 7, 30, 3)])
def test_matches_spin_orbital_density(o, v, naux, seed):
    eps_o, eps_v, Bov = draw(o, v, naux, seed)
    r = M.mp2_bno(eps_o, eps_v, Bov)
    goo, gvv = spin_orbital_density(eps_o, eps_v, r["ovov"])
    np.testing.assert_allclose(r["gamma_oo"], goo, rtol=0, atol=1e-14)
    np.testing.assert_allclose(r["gamma_vv"], gvv, rtol=0, atol=1e-15 * max(1.0, np.abs(gvv).max()))


@pytest.mark.parametrize("o,v,naux,seed", [(3, 9, 48, 4), (6, 40, 184, 5), (8, 64, 288, 6)])
def test_particle_number_symmetry_and_populations(o, v, naux, seed):
    eps_o, eps_v, Bov = draw(o, v, naux, seed)
    r = M.mp2_bno(eps_o, eps_v, Bov)
    assert abs(np.trace(r["gamma_oo"]) + np.trace(r["gamma_vv"]) - 2 * o) <= 1e-12 * o
    for g in (r["gamma_oo"], r["gamma_vv"]):
        np.testing.assert_allclose(g, g.T, rtol=0, atol=1e-15)
    for g, p in ((r["gamma_oo"], r["pop_o"]), (r["gamma_vv"], r["pop_v"])):
        assert np.all(np.diff(p) >= 0.0)
        assert abs(p.sum() - np.trace(g)) <= 1e-12 * max(1.0, abs(np.trace(g)))
        sign, logdet = np.linalg.slogdet(g)
        assert sign > 0 and abs(np.sum(np.log(p)) - logdet) <= 1e-9 * abs(logdet) + 1e-9
    # occupied populations just below 2, virtual ones small and positive
    assert np.all(r["pop_o"] < 2.0) and np.all(r["pop_o"] > 1.5)
    assert np.all(r["pop_v"] > 0.0) and np.all(r["pop_v"] < 0.5)


def test_relabelling_invariance():
    eps_o, eps_v, Bov = draw(5, 17, 88, 7)
    r = M.mp2_bno(eps_o, eps_v, Bov)
    rng = np.random.default_rng(7)
    po, pv = rng.permutation(5), rng.permutation(17)
    s = M.mp2_bno(eps_o[po], eps_v[pv], Bov[:, po][:, :, pv])
    np.testing.assert_allclose(s["pop_o"], r["pop_o"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(s["pop_v"], r["pop_v"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(s["gamma_vv"], r["gamma_vv"][np.ix_(pv, pv)], rtol=0, atol=1e-16)


def test_uncorrelated_limit():
    eps_o, eps_v, Bov = draw(3, 8, 40, 8)
    r = M.mp2_bno(eps_o, eps_v, 0.0 * Bov)
    np.testing.assert_array_equal(r["gamma_oo"], 2.0 * np.eye(3))
    np.testing.assert_array_equal(r["gamma_vv"], np.zeros((8, 8)))


def test_planted_mistakes_break_a_pin(monkeypatch):
    eps_o, eps_v, Bov = draw(3, 5, 20, 2)
    ovov = M.ovov_from_df(Bov)
    goo_s, gvv_s = spin_orbital_density(eps_o, eps_v, ovov)

    def bad_exchange_vv(t2):  # + instead of - in the exchange term
        return 2.0 * np.einsum("ijac,ijbc->ab", t2, 2.0 * t2 + np.einsum("ijbc->ijcb", t2))

    def bad_factor_vv(t2):    # the leading 2 dropped
        return np.einsum("ijac,ijbc->ab", t2, 2.0 * t2 - np.einsum("ijbc->ijcb", t2))

    for bad in (bad_exchange_vv, bad_factor_vv):
        monkeypatch.setattr(M, "rdm1_vv", bad)
        r = M.mp2_bno(eps_o, eps_v, Bov)
        assert np.abs(r["gamma_vv"] - gvv_s).max() > 1e-6
    monkeypatch.undo()
    # an amplitude sign error leaves the density (quadratic in t) unchanged but
    # not the amplitudes' relation to the integrals: t (ia|jb) summed is negative
    r = M.mp2_bno(eps_o, eps_v, Bov)
    assert np.einsum("ijab,iajb->", r["t2"], ovov) < 0.0
