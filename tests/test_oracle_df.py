"""Pins of the density-fitted (ov|vv) oracle (oracle/df.py) against what the
definition fixes, independently of its own code:

* brute force: every entry as an explicit sum over P on a tiny cluster;
* the generator's whole integral tensor (pq|rs) over all orbitals, formed by a
  different route (one matrix product of the flattened factor), restricted to
  its (ov|vv) block;
* the (b, d) symmetry that a symmetric factor (B[P,p,q] = B[P,q,p]) implies;
* a planted mistake (the two virtual indices of Bvv swapped in a
  non-symmetric factor, a transposed Bov) breaks the brute-force pin."""
import itertools

import numpy as np

import tegen
from oracle import df as D


def factors(o, v, naux, seed):
    c = tegen.make_cluster(o, v, naux, seed, with_df=True)
    return c, c.Bov, c.Bvv


def test_brute_force():
    rng = np.random.default_rng(3)
    naux, o, v = 5, 2, 3
    Bov, Bvv = rng.standard_normal((naux, o, v)), rng.standard_normal((naux, v, v))
    got = D.ovvv_from_df(Bov, Bvv)
    for i, a, b, d in itertools.product(range(o), range(v), range(v), range(v)):
        ref = 0.0
        for P in range(naux):
            ref += Bov[P, i, a] * Bvv[P, b, d]
        assert abs(got[i, a, b, d] - ref) <= 1e-15 * max(1.0, abs(ref))


def test_matches_full_integrals_and_generator():
    o, v, naux, seed = 3, 7, 30, 5
    c, Bov, Bvv = factors(o, v, naux, seed)
    eri = tegen.eri_full(o, v, naux, seed)
    got = D.ovvv_from_df(Bov, Bvv)
    np.testing.assert_allclose(got, eri[:o, o:, o:, o:], rtol=0, atol=1e-16)
    np.testing.assert_allclose(got, c.ovvv, rtol=0, atol=1e-16)


def test_virtual_pair_symmetry():
    _, Bov, Bvv = factors(4, 9, 40, 6)
    got = D.ovvv_from_df(Bov, Bvv)
    np.testing.assert_allclose(got, got.transpose(0, 1, 3, 2), rtol=0, atol=1e-17)


def test_planted_mistakes_break_the_pin():
    rng = np.random.default_rng(4)
    Bov, Bvv = rng.standard_normal((6, 2, 3)), rng.standard_normal((6, 3, 3))
    ref = np.zeros((2, 3, 3, 3))
    for i, a, b, d in itertools.product(range(2), range(3), range(3), range(3)):
        ref[i, a, b, d] = sum(Bov[P, i, a] * Bvv[P, b, d] for P in range(6))
    swapped = np.einsum("Pia,Pdb->iabd", Bov, Bvv)
    assert np.abs(swapped - ref).max() > 1e-3
    Bsq = rng.standard_normal((6, 3, 3))
    transposed = np.einsum("Pai,Pbd->iabd", Bsq, Bvv)[:3, :3]
    ref_sq = np.einsum("Pia,Pbd->iabd", Bsq, Bvv)
    assert np.abs(transposed - ref_sq).max() > 1e-3
