"""FP64 CPU oracle for the MP2 step that precedes (T) in the SIE workflow:
subspace MP2 amplitudes, the MP2 one-body reduced density matrix and the
bath-natural-orbital (BNO) populations, from the supplement section on
BNO construction (the MP2 amplitude, denominator and 1-RDM equations there).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only
the tests and ``bench.py``'s cpu_baseline leg may.  Plain float64 numpy, with
``numpy.einsum`` for the contractions and ``numpy.linalg.eigvalsh`` for the
diagonalisation (library primitives); no blocking or fusion.  It shares no
code with the CUDA path.

Per cluster, with the density-fitting factor of the occupied-virtual block
B[P, i, a] (chemists' notation, (ia|jb) = sum_P B[P,i,a] B[P,j,b]):

* t_ij^ab = -(ia|jb) / D_ij^ab,  D_ij^ab = e_a + e_b - e_i - e_j;
* gamma_ab = 2 sum_ij sum_c t_ij^ac (2 t_ij^bc - t_ij^cb)        (virtual block);
* gamma_ij = 2 delta_ij - 2 sum_k sum_ab t_ik^ab (2 t_jk^ab - t_jk^ba)   (occupied);
* the occupied-virtual block of the MP2 1-RDM is zero;
* BNO populations: the eigenvalues of each block (ascending).

Array conventions (float64, row-major): eps_o[o], eps_v[v], Bov[P][o][v],
ovov[i,a,j,b] = (ia|jb), t2[i,j,a,b] = t_ij^ab, gamma_vv[v][v], gamma_oo[o][o].
"""
from __future__ import annotations

import numpy as np


def ovov_from_df(Bov):
    """(ia|jb) = sum_P B[P,i,a] B[P,j,b], indexed [i,a,j,b]."""
    return np.einsum("Pia,Pjb->iajb", Bov, Bov)


def mp2_denominator(eps_o, eps_v):
    """D_ij^ab = e_a + e_b - e_i - e_j, indexed [i,j,a,b]."""
    return (eps_v[None, None, :, None] + eps_v[None, None, None, :]
            - eps_o[:, None, None, None] - eps_o[None, :, None, None])


def mp2_amplitudes(eps_o, eps_v, ovov):
    """t_ij^ab = -(ia|jb) / D_ij^ab, indexed [i,j,a,b]."""
    return -np.einsum("iajb->ijab", ovov) / mp2_denominator(eps_o, eps_v)


def rdm1_vv(t2):
    """gamma_ab = 2 sum_ij sum_c t_ij^ac (2 t_ij^bc - t_ij^cb)."""
    tt = 2.0 * t2 - np.einsum("ijbc->ijcb", t2)
    return 2.0 * np.einsum("ijac,ijbc->ab", t2, tt)


def rdm1_oo(t2):
    """gamma_ij = 2 delta_ij - 2 sum_k sum_ab t_ik^ab (2 t_jk^ab - t_jk^ba)."""
    o = t2.shape[0]
    tt = 2.0 * t2 - np.einsum("jkba->jkab", t2)
    return 2.0 * np.eye(o) - 2.0 * np.einsum("ikab,jkab->ij", t2, tt)


def populations(gamma):
    """BNO populations: the eigenvalues of a 1-RDM block, ascending."""
    return np.linalg.eigvalsh(gamma)


def mp2_bno(eps_o, eps_v, Bov):
    """Everything for one cluster: dict of ovov, t2, gamma_oo, gamma_vv,
    pop_o, pop_v."""
    eps_o = np.asarray(eps_o, dtype=np.float64)
    eps_v = np.asarray(eps_v, dtype=np.float64)
    ovov = ovov_from_df(np.asarray(Bov, dtype=np.float64))
    t2 = mp2_amplitudes(eps_o, eps_v, ovov)
    goo, gvv = rdm1_oo(t2), rdm1_vv(t2)
    return dict(ovov=ovov, t2=t2, gamma_oo=goo, gamma_vv=gvv, pop_o=populations(goo), pop_v=populations(gvv))
