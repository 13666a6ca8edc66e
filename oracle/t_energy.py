"""FP64 CPU oracle for the closed-shell perturbative-triples energy E(T).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only
the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg
of ``bench.py`` may.  It is a plain, slow transcription of the formula in the
supplement section "The In-situ Form of Perturbative (T) in SIE", written in
plain PyTorch CPU ops in float64, with ``torch.einsum`` as the only library
primitive (contractions and index permutations).  It shares no code with the
CUDA path.

Formula (C^f = identity, i.e. the whole-cluster (T)):

* Eq. (E_corr_CCSD_T):  E = 2 sum_{a>=b>=c} sum_{ijk} A R[Z]_{ijk}^{abc} W~_{ijk}^{abc}
  with A = 1/6 (a=b=c), 1/2 (a=b or b=c), 1 otherwise;
* Z = W + V, with W = P[X]/D (Eq. W_in_CCSD_T) and V = 1/2 P[(ia|jb) t_k^c]/D
  (Eq. V_in_CCSD_T), so that Z = (W~ + Y)/D with W~ = W D and Y = 1/2 P[(ia|jb) t_k^c];
* D = e_i + e_j + e_k - e_a - e_b - e_c;
* P[X]^{abc}_{ijk} = X^{abc}_{ijk} + X^{bca}_{jki} + X^{cab}_{kij} + X^{acb}_{ikj}
  + X^{cba}_{kji} + X^{bac}_{jik};
* R[X]_{ijk} = 4 X_{ijk} + X_{kij} + X_{jki} - 2 X_{kji} - 2 X_{ikj} - 2 X_{jik}
  (fixed abc).

With a general C^f (``t_energy_projected``): the first occupied index of W~
is projected, E_x = (1/3) sum_{ijk} sum_{abc} sum_{i'} C^f_{ii'} W~_{i'jk} R[Z]_{ijk}
over all ordered triples; at C^f = 1 this is the restricted sum below, and
for a general C^f the literal restricted sum would depend on the labelling of
the virtual orbitals, so the full sum is the reading.  Pinned by
tests/test_oracle_projected.py (identity, partition of unity, slot
independence, shares, linearity).

Readings where the printed text is garbled (each is listed in the design notes):

* the bracket of Eq. W is read as  sum_d (ia|bd) t_{kj}^{cd} - sum_l (ia|jl) t_{lk}^{bc}
  (the printed text swaps the dummy indices l and d);
* the R operator's ``X_{klj}`` is read as ``X_{kij}`` (the second cyclic permutation);
* the restriction "(ia >= jb >= kc)" with A depending on a, b, c is read as
  a >= b >= c over virtuals with all i, j, k;
* there is no f_ov t2 term in V (canonical orbitals, no Fock matrix in the interface).

Array conventions (all float64, row-major): eps_o[o], eps_v[v],
ovvv[i,a,b,d] = (ia|bd), ooov[j,l,i,a] = (jl|ia) = (ia|jl), ovov[i,a,j,b] = (ia|jb),
t1[i,a] = t_i^a, t2[i,j,a,b] = t_{ij}^{ab}.  No symmetry of the inputs is assumed.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np
import torch

NAMES = ("eps_o", "eps_v", "ovvv", "ooov", "ovov", "t1", "t2")


@dataclass
class Inputs:
    eps_o: torch.Tensor
    eps_v: torch.Tensor
    ovvv: torch.Tensor
    ooov: torch.Tensor
    ovov: torch.Tensor
    t1: torch.Tensor
    t2: torch.Tensor

    @property
    def nocc(self):
        return self.eps_o.shape[0]

    @property
    def nvir(self):
        return self.eps_v.shape[0]


def inputs(eps_o, eps_v, ovvv, ooov, ovov, t1, t2, requires_grad=False) -> Inputs:
    """Wrap seven arrays (numpy or torch) as CPU float64 tensors."""
    def conv(x):
        if isinstance(x, torch.Tensor):
            t = x.detach().to("cpu", torch.float64).clone()
        else:
            t = torch.from_numpy(np.array(x, dtype=np.float64, copy=True))
        return t.requires_grad_(requires_grad)
    return Inputs(*(conv(x) for x in (eps_o, eps_v, ovvv, ooov, ovov, t1, t2)))


# ---------------------------------------------------------------------------
# Building blocks, one per printed quantity
# ---------------------------------------------------------------------------

def x_bracket(c: Inputs, p, q, r):
    """The bracket of Eq. (W_in_CCSD_T) at occupied (p,q,r), over all virtuals:
    X_{pqr}^{abc} = sum_d (pa|bd) t_{rq}^{cd} - sum_l (pa|ql) t_{lr}^{bc}."""
    vvvo = torch.einsum("abd,cd->abc", c.ovvv[p], c.t2[r, q])
    ooov = torch.einsum("la,lbc->abc", c.ooov[q, :, p, :], c.t2[:, r])
    return vvvo - ooov


def sym_p(f, i, j, k):
    """The permutation operator P of the section: f(p,q,r) returns an array
    indexed [alpha,beta,gamma] = X^{alpha beta gamma}_{pqr}; the result is
    P[X]^{abc}_{ijk} as an array indexed [a,b,c]."""
    return (f(i, j, k)                                    # X^{abc}_{ijk}
            + torch.einsum("bca->abc", f(j, k, i))        # X^{bca}_{jki}
            + torch.einsum("cab->abc", f(k, i, j))        # X^{cab}_{kij}
            + torch.einsum("acb->abc", f(i, k, j))        # X^{acb}_{ikj}
            + torch.einsum("cba->abc", f(k, j, i))        # X^{cba}_{kji}
            + torch.einsum("bac->abc", f(j, i, k)))       # X^{bac}_{jik}


def w_tilde(c: Inputs, i, j, k):
    """W~_{ijk}^{abc} = W D = P[X] (Eq. W_in_CCSD_T and the definition of W~)."""
    return sym_p(lambda p, q, r: x_bracket(c, p, q, r), i, j, k)


def y_disconnected(c: Inputs, i, j, k):
    """Y_{ijk}^{abc} = V D = 1/2 P[(ia|jb) t_k^c]  (Eq. V_in_CCSD_T)."""
    def u(p, q, r):
        return torch.einsum("ab,c->abc", c.ovov[p, :, q, :], c.t1[r])
    return 0.5 * sym_p(u, i, j, k)


def denominator(c: Inputs, i, j, k):
    """D_{ijk}^{abc} = e_i + e_j + e_k - e_a - e_b - e_c, indexed [a,b,c]."""
    ev = c.eps_v
    eo = c.eps_o[i] + c.eps_o[j] + c.eps_o[k]
    return eo - ev[:, None, None] - ev[None, :, None] - ev[None, None, :]


def r_operator(x):
    """R[X]_{ijk} at fixed abc (Eq. R_opt_in_CCSD(T), reading X_{klj} -> X_{kij}).
    ``x`` maps an occupied ordering (p,q,r) to X_{pqr} (an array over abc) and is
    called with the orderings of (i,j,k) = ``x.ijk``.  The terms are grouped
    (4X - 2X - 2X) + (X + X - 2X) so that R vanishes exactly when i = j = k."""
    i, j, k = x.ijk
    return ((4.0 * x(i, j, k) - 2.0 * x(k, j, i) - 2.0 * x(i, k, j))
            + (x(k, i, j) + x(j, k, i) - 2.0 * x(j, i, k)))


class _ByOrdering:
    def __init__(self, ijk, fn):
        self.ijk = ijk
        self._fn = fn
        self._cache = {}

    def __call__(self, p, q, r):
        key = (p, q, r)
        if key not in self._cache:
            self._cache[key] = self._fn(p, q, r)
        return self._cache[key]


# ---------------------------------------------------------------------------
# Energies
# ---------------------------------------------------------------------------

def triple_energy(c: Inputs, i, j, k):
    """e_{ijk} = sum_{abc} W~_{ijk}^{abc} R[Z]_{ijk}^{abc}, Z = (W~ + Y)/D, for one
    ordered occupied triple, summed over all virtual triples.  Every ordering of
    (i,j,k) that R needs is built from the formula (no symmetry shortcut)."""
    z = _ByOrdering((i, j, k), lambda p, q, r:
                    (w_tilde(c, p, q, r) + y_disconnected(c, p, q, r))
                    / denominator(c, p, q, r))
    return (w_tilde(c, i, j, k) * r_operator(z)).sum()


def triple_multiplicity(i, j, k):
    """Number of distinct orderings of (i,j,k)."""
    return len(set(itertools.permutations((i, j, k))))


def unique_triples(nocc):
    """i >= j >= k with i = j = k left out, lexicographic in (i, j, k).  This is
    the order of the per-triple energies of the library's triple-range call."""
    return [(i, j, k) for i in range(nocc) for j in range(i + 1)
            for k in range(j + 1) if not (i == j == k)]


def triple_share(c: Inputs, i, j, k):
    """The energy share of the unique triple {i,j,k}: (m/3) e_{ijk}, m the number
    of distinct orderings.  Summed over all unique triples this is E (the
    restricted sum of Eq. E_corr_CCSD_T equals one third of the unrestricted sum
    over all abc and all ordered ijk)."""
    return triple_multiplicity(i, j, k) / 3.0 * triple_energy(c, i, j, k)


def t_energy(c: Inputs, triples=None):
    """E(T) as the sum of the unique-triple shares (float64 scalar tensor)."""
    if triples is None:
        triples = unique_triples(c.nocc)
    total = torch.zeros((), dtype=torch.float64)
    for (i, j, k) in triples:
        total = total + triple_share(c, i, j, k)
    return total


def t_energy_ordered(c: Inputs):
    """E(T) = (1/3) sum over all ordered triples ijk of e_{ijk} (no use of the
    invariance of e under reordering of ijk)."""
    o = c.nocc
    total = torch.zeros((), dtype=torch.float64)
    for i in range(o):
        for j in range(o):
            for k in range(o):
                total = total + triple_energy(c, i, j, k)
    return total / 3.0


def t_energy_restricted(c: Inputs):
    """Eq. (E_corr_CCSD_T) literally: 2 sum_{a>=b>=c} A sum_{ijk} R[Z] W~, with all
    six-index arrays held in memory (tiny clusters only)."""
    o, v = c.nocc, c.nvir
    Wt = torch.stack([torch.stack([torch.stack([w_tilde(c, i, j, k) for k in range(o)])
                                   for j in range(o)]) for i in range(o)])
    Y = torch.stack([torch.stack([torch.stack([y_disconnected(c, i, j, k) for k in range(o)])
                                  for j in range(o)]) for i in range(o)])
    D = torch.stack([torch.stack([torch.stack([denominator(c, i, j, k) for k in range(o)])
                                  for j in range(o)]) for i in range(o)])
    Z = (Wt + Y) / D
    RZ = ((4.0 * Z - 2.0 * torch.einsum("kjiabc->ijkabc", Z) - 2.0 * torch.einsum("ikjabc->ijkabc", Z))
          + (torch.einsum("kijabc->ijkabc", Z) + torch.einsum("jkiabc->ijkabc", Z)
             - 2.0 * torch.einsum("jikabc->ijkabc", Z)))
    a = torch.arange(v)
    ge = (a[:, None, None] >= a[None, :, None]) & (a[None, :, None] >= a[None, None, :])
    eq_ab = a[:, None, None] == a[None, :, None]
    eq_bc = a[None, :, None] == a[None, None, :]
    A = torch.where(eq_ab & eq_bc, 1.0 / 6.0,
                    torch.where(eq_ab | eq_bc, 0.5, 1.0)).to(torch.float64)
    A = torch.where(ge, A, torch.zeros((), dtype=torch.float64))
    return 2.0 * (A[None, None, None] * RZ * Wt).sum()


# ---------------------------------------------------------------------------
# Fragment-projected energy: Eq. (E_corr_CCSD_T) with a general C^f
# ---------------------------------------------------------------------------
#
# E_x = 2 sum_{(ia>=jb>=kc)} sum_{i'} A R[Z]_{ijk} W~_{i'jk} C^f_{ii'}: the first
# occupied index of W~ is projected.  Reading: the sum is the full one,
# E_x = (1/3) sum_{ijk} sum_{abc} sum_{i'} C^f_{ii'} W~_{i'jk} R[Z]_{ijk}, which is
# the printed restricted sum when C^f = 1.  For a general C^f the restricted
# sum over a >= b >= c depends on how the virtual orbitals are labelled (the
# summand is no longer symmetric under joint permutations of abc and ijk), the
# full sum does not.

def project_first(cf, wt, j, k):
    """sum_{i'} cf[i, i'] W~_{i'jk} for every i, as an array [i, a, b, c];
    ``wt(p, q, r)`` returns W~_{pqr}."""
    o = cf.shape[0]
    stack = torch.stack([wt(p, j, k) for p in range(o)])
    return torch.einsum("ip,pabc->iabc", cf, stack)


def _blocks(c: Inputs):
    """W~ and Z = (W~ + Y)/D of every ordered triple, built on demand and kept."""
    wt_cache, z_cache = {}, {}

    def wt(p, q, r):
        if (p, q, r) not in wt_cache:
            wt_cache[(p, q, r)] = w_tilde(c, p, q, r)
        return wt_cache[(p, q, r)]

    def z(p, q, r):
        if (p, q, r) not in z_cache:
            z_cache[(p, q, r)] = (wt(p, q, r) + y_disconnected(c, p, q, r)) / denominator(c, p, q, r)
        return z_cache[(p, q, r)]
    return wt, z


def triple_energy_projected(c: Inputs, cf, i, j, k, blocks=None, slot=0):
    """e^f_{ijk} = sum_{abc} sum_{i'} cf[i,i'] W~_{i'jk} R[Z]_{ijk} for one ordered
    triple.  ``slot`` = 1 or 2 projects the second or third occupied index of
    W~ instead (the same total after the sum over all ordered triples)."""
    wt, z = blocks if blocks is not None else _blocks(c)
    zz = _ByOrdering((i, j, k), z)
    rz = r_operator(zz)
    ijk = (i, j, k)
    o = cf.shape[0]
    wp = torch.zeros_like(rz)
    for p in range(o):
        idx = list(ijk)
        idx[slot] = p
        wp = wp + cf[ijk[slot], p] * wt(*idx)
    return (wp * rz).sum()


def t_energy_projected(c: Inputs, cf, slot=0):
    """E_x = (1/3) sum over all ordered triples of e^f_{ijk} (float64 scalar)."""
    cf = torch.as_tensor(np.asarray(cf), dtype=torch.float64)
    blocks = _blocks(c)
    o = c.nocc
    total = torch.zeros((), dtype=torch.float64)
    for i in range(o):
        for j in range(o):
            for k in range(o):
                total = total + triple_energy_projected(c, cf, i, j, k, blocks, slot)
    return total / 3.0


def triple_share_projected(c: Inputs, cf, i, j, k, blocks=None):
    """The share of the unique triple {i,j,k}: (1/3) sum over its distinct
    orderings of e^f.  Summed over the unique triples this is E_x."""
    cf = torch.as_tensor(np.asarray(cf), dtype=torch.float64)
    blocks = blocks if blocks is not None else _blocks(c)
    total = torch.zeros((), dtype=torch.float64)
    for perm in set(itertools.permutations((i, j, k))):
        total = total + triple_energy_projected(c, cf, *perm, blocks)
    return total / 3.0


def t_energy_projected_restricted(c: Inputs, cf):
    """The printed restricted form taken literally with a general C^f:
    2 sum_{a>=b>=c} A sum_{ijk} sum_{i'} R[Z]_{ijk} W~_{i'jk} C^f_{ii'} (tiny
    clusters; kept to show why the full sum is the reading)."""
    o, v = c.nocc, c.nvir
    cf = torch.as_tensor(np.asarray(cf), dtype=torch.float64)
    wt, z = _blocks(c)
    Wt = torch.stack([torch.stack([torch.stack([wt(i, j, k) for k in range(o)])
                                   for j in range(o)]) for i in range(o)])
    Z = torch.stack([torch.stack([torch.stack([z(i, j, k) for k in range(o)])
                                  for j in range(o)]) for i in range(o)])
    RZ = ((4.0 * Z - 2.0 * torch.einsum("kjiabc->ijkabc", Z) - 2.0 * torch.einsum("ikjabc->ijkabc", Z))
          + (torch.einsum("kijabc->ijkabc", Z) + torch.einsum("jkiabc->ijkabc", Z)
             - 2.0 * torch.einsum("jikabc->ijkabc", Z)))
    WP = torch.einsum("ip,pjkabc->ijkabc", cf, Wt)
    a = torch.arange(v)
    ge = (a[:, None, None] >= a[None, :, None]) & (a[None, :, None] >= a[None, None, :])
    eq_ab = a[:, None, None] == a[None, :, None]
    eq_bc = a[None, :, None] == a[None, None, :]
    A = torch.where(eq_ab & eq_bc, 1.0 / 6.0,
                    torch.where(eq_ab | eq_bc, 0.5, 1.0)).to(torch.float64)
    A = torch.where(ge, A, torch.zeros((), dtype=torch.float64))
    return 2.0 * (A[None, None, None] * RZ * WP).sum()


# ---------------------------------------------------------------------------
# Gradient
# ---------------------------------------------------------------------------

def t_energy_grad(c: Inputs, triples=None):
    """dE/d(eps_o, eps_v, ovvv, ooov, ovov, t1, t2): the derivative of E with
    every stored entry an independent variable, by reverse-mode differentiation
    of ``t_energy`` one triple at a time.  Returns (E, dict of gradients)."""
    leaves = inputs(*(getattr(c, n) for n in NAMES), requires_grad=True)
    if triples is None:
        triples = unique_triples(leaves.nocc)
    e = 0.0
    for (i, j, k) in triples:
        share = triple_share(leaves, i, j, k)
        share.backward()
        e += float(share.detach())
    grads = {}
    for n in NAMES:
        g = getattr(leaves, n).grad
        grads[n] = torch.zeros_like(getattr(leaves, n)) if g is None else g.detach()
    return e, grads
