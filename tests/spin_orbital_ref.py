"""Spin-orbital (T) energy: an independent formulation used to pin the oracle.

The closed-shell formula the oracle transcribes is a spin adaptation of the
general spin-orbital (T) correction (Raghavachari, Trucks, Pople, Head-Gordon
1989; spin-orbital working equations as in Crawford & Schaefer, Rev. Comp.
Chem. 14 (2000)):

    D t_c(ijk,abc) = P(i/jk) P(a/bc) [ sum_e t_jk^ae <ei||bc> - sum_m t_im^bc <ma||jk> ]
    D t_d(ijk,abc) = P(i/jk) P(a/bc) t_i^a <jk||bc>
    E(T) = (1/36) sum_{ijkabc} t_c D (t_c + t_d)

with P(i/jk) f(ijk) = f(ijk) - f(jik) - f(kji), antisymmetrised physicists'
integrals <pq||rs> = (pr|qs) - (ps|qr) and D = e_i + e_j + e_k - e_a - e_b - e_c.
It shares nothing with the closed-shell form but the inputs: spin-adapted
amplitudes of a closed-shell reference, real integrals with 8-fold symmetry.
Tiny clusters only (six-index spin-orbital arrays).
"""
import numpy as np


def spin_orbital_t_energy(eri, nocc, eps_o, eps_v, t1, t2):
    n = eri.shape[0]
    nvir = n - nocc
    so = 2 * nocc
    sv = 2 * nvir
    spat_o = np.repeat(np.arange(nocc), 2)
    spin_o = np.tile([0, 1], nocc)
    spat_v = np.repeat(np.arange(nvir), 2)
    spin_v = np.tile([0, 1], nvir)
    spat = np.concatenate([spat_o, nocc + spat_v])
    spin = np.concatenate([spin_o, spin_v])
    # <PQ|RS> = (pr|qs) d(sP,sR) d(sQ,sS)
    same = (spin[:, None] == spin[None, :]).astype(float)
    phys = (eri[np.ix_(spat, spat, spat, spat)].transpose(0, 2, 1, 3)
            * same[:, None, :, None] * same[None, :, None, :])
    g = phys - phys.transpose(0, 1, 3, 2)
    O = slice(0, so)
    V = slice(so, so + sv)

    T1 = t1[np.ix_(spat_o, spat_v)] * (spin_o[:, None] == spin_v[None, :])
    d = lambda x, y: (x[:, None] == y[None, :]).astype(float)
    T2 = (t2[np.ix_(spat_o, spat_o, spat_v, spat_v)]
          * d(spin_o, spin_v)[:, None, :, None] * d(spin_o, spin_v)[None, :, None, :]
          - t2[np.ix_(spat_o, spat_o, spat_v, spat_v)].transpose(0, 1, 3, 2)
          * d(spin_o, spin_v)[:, None, None, :] * d(spin_o, spin_v)[None, :, :, None])

    f = (np.einsum("jkae,eibc->ijkabc", T2, g[V, O, V, V])
         - np.einsum("imbc,majk->ijkabc", T2, g[O, V, O, O]))
    fd = np.einsum("ia,jkbc->ijkabc", T1, g[O, O, V, V])

    def perm(x):
        x = x - x.transpose(1, 0, 2, 3, 4, 5) - x.transpose(2, 1, 0, 3, 4, 5)
        return x - x.transpose(0, 1, 2, 4, 3, 5) - x.transpose(0, 1, 2, 5, 4, 3)

    Wc = perm(f)
    Vd = perm(fd)
    eo = eps_o[spat_o]
    ev = eps_v[spat_v]
    D = (eo[:, None, None, None, None, None] + eo[None, :, None, None, None, None]
         + eo[None, None, :, None, None, None] - ev[None, None, None, :, None, None]
         - ev[None, None, None, None, :, None] - ev[None, None, None, None, None, :])
    return float((Wc * (Wc + Vd) / D).sum() / 36.0)
