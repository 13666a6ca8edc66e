"""Pins of the oracle's fragment-projected energy (Eq. E_corr_CCSD_T with a
general C^f, the first occupied index of W~ projected), each against a fact
the definition fixes independently of how the oracle computes it:

* C^f = 1 gives the whole-cluster energy (three independent forms of it);
* projectors of a partition of the occupied space sum to the whole-cluster
  energy (linearity of Eq. C_f in C^f and sum_x C^{f_x} = 1);
* projecting the second or third occupied index of W~ instead gives the same
  total (the symmetry the GPU path relies on);
* unique-triple shares add up to the total; i = j = k contributes nothing;
* the printed restricted sum taken literally depends on the labelling of
  the virtual orbitals when C^f != 1, the full sum does not (the reading)."""
import numpy as np
import pytest
import torch

import tegen
from oracle import t_energy as O


@pytest.fixture(scope="module")
def cluster():
    a = tegen.make_cluster(4, 7, 44, 3).arrays()
    a["t1"] = a["t1"] * 50.0
    return a


def _orthogonal(o, seed):
    u, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((o, o)))
    return u


def test_identity_projector_is_the_cluster_energy(cluster):
    c = O.inputs(**cluster)
    e = float(O.t_energy(c))
    ef = float(O.t_energy_projected(c, np.eye(c.nocc)))
    er = float(O.t_energy_projected_restricted(c, np.eye(c.nocc)))
    assert abs(ef - e) <= 1e-12 * abs(e)
    assert abs(er - e) <= 1e-12 * abs(e)


@pytest.mark.parametrize("split", [(2, 2), (1, 3), (1, 1, 2)])
def test_partition_of_unity(cluster, split):
    c = O.inputs(**cluster)
    u = _orthogonal(c.nocc, sum(split))
    e = float(O.t_energy(c))
    total, col = 0.0, 0
    for n in split:
        f = u[:, col:col + n]
        col += n
        total += float(O.t_energy_projected(c, f @ f.T))
    assert abs(total - e) <= 1e-11 * abs(e)


def test_projecting_another_slot_gives_the_same_total(cluster):
    c = O.inputs(**cluster)
    cf = np.random.default_rng(7).standard_normal((c.nocc, c.nocc))  # not symmetric
    e0 = float(O.t_energy_projected(c, cf, slot=0))
    for slot in (1, 2):
        assert abs(float(O.t_energy_projected(c, cf, slot=slot)) - e0) <= 1e-12 * abs(e0)


def test_shares_add_up_and_diagonal_triples_vanish(cluster):
    c = O.inputs(**cluster)
    cf = np.random.default_rng(8).standard_normal((c.nocc, c.nocc))
    cf = cf + cf.T
    blocks = O._blocks(c)
    cft = torch.as_tensor(cf)
    shares = [float(O.triple_share_projected(c, cf, *t, blocks)) for t in O.unique_triples(c.nocc)]
    e = float(O.t_energy_projected(c, cf))
    assert abs(sum(shares) - e) <= 1e-12 * abs(e)
    for i in range(c.nocc):
        assert float(O.triple_energy_projected(c, cft, i, i, i, blocks)) == 0.0


def test_linear_in_the_projector(cluster):
    c = O.inputs(**cluster)
    rng = np.random.default_rng(9)
    c1, c2 = rng.standard_normal((2, c.nocc, c.nocc))
    lhs = float(O.t_energy_projected(c, 2.0 * c1 - 0.5 * c2))
    rhs = 2.0 * float(O.t_energy_projected(c, c1)) - 0.5 * float(O.t_energy_projected(c, c2))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_restricted_literal_form_depends_on_virtual_labels(cluster):
    """Why the full sum is the reading: relabelling the virtual orbitals leaves
    the full sum unchanged and changes the literal restricted one."""
    c = O.inputs(**cluster)
    u = _orthogonal(c.nocc, 0)
    cf = u[:, :2] @ u[:, :2].T
    pv = np.random.default_rng(5).permutation(c.nvir)
    a = cluster
    b = dict(eps_o=a["eps_o"], eps_v=a["eps_v"][pv],
             ovvv=a["ovvv"][:, pv][:, :, pv][:, :, :, pv], ooov=a["ooov"][:, :, :, pv],
             ovov=a["ovov"][:, pv][:, :, :, pv], t1=a["t1"][:, pv], t2=a["t2"][:, :, pv][:, :, :, pv])
    cb = O.inputs(**{k: np.ascontiguousarray(x) for k, x in b.items()})
    full, full_b = float(O.t_energy_projected(c, cf)), float(O.t_energy_projected(cb, cf))
    assert abs(full - full_b) <= 1e-12 * abs(full)
    lit, lit_b = float(O.t_energy_projected_restricted(c, cf)), float(O.t_energy_projected_restricted(cb, cf))
    assert abs(lit - lit_b) > 1e-3 * abs(lit)
