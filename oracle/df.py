"""FP64 CPU oracle for the (ov|vv) integrals of a density-fitted cluster.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only
the tests and ``bench.py`` may.  Plain float64 numpy (``numpy.einsum``, a
library primitive); it shares no code with the CUDA path.

The clusters' integrals are density-fitted, (pq|rs) = sum_P B[P,p,q]
B[P,r,s] in chemists' notation.  E(T) reads the (ov|vv) block

    ovvv[i,a,b,d] = (ia|bd) = sum_P Bov[P,i,a] Bvv[P,b,d]

with Bov = B[:, occupied, virtual] and Bvv = B[:, virtual, virtual].  The
supplement's remark on the divisibility of the (T) contraction (the energy
never needs a whole six-index tensor) is what lets a GPU code form these
slabs on the fly; the oracle forms the whole block, then calls the (T)
oracle (``oracle.t_energy``) on it.
"""
from __future__ import annotations

import numpy as np


def ovvv_from_df(Bov, Bvv):
    """(ia|bd) = sum_P Bov[P,i,a] Bvv[P,b,d], indexed [i,a,b,d]."""
    return np.einsum("Pia,Pbd->iabd", np.asarray(Bov, dtype=np.float64), np.asarray(Bvv, dtype=np.float64))
