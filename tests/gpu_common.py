"""Helpers shared by the GPU test modules."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def golden(name):
    with open(os.path.join(HERE, "golden", f"oracle_{name}.json")) as f:
        return json.load(f)


def check_inputs_match(cl, g, rtol=1e-12):
    for n, (s, sa) in g["checksums"].items():
        a = cl.arrays()[n]
        assert abs(float(np.sum(np.abs(a))) - sa) <= rtol * sa, f"generator drew different {n}"


def shuffled(arrs, seed):
    """Relabel occupied and virtual orbitals: orbital energies become unsorted."""
    rng = np.random.default_rng(seed)
    o, v = arrs["t1"].shape
    po, pv = rng.permutation(o), rng.permutation(v)
    a = arrs
    return dict(eps_o=a["eps_o"][po], eps_v=a["eps_v"][pv],
                ovvv=np.ascontiguousarray(a["ovvv"][np.ix_(po, pv, pv, pv)]),
                ooov=np.ascontiguousarray(a["ooov"][np.ix_(po, po, po, pv)]),
                ovov=np.ascontiguousarray(a["ovov"][np.ix_(po, pv, po, pv)]),
                t1=np.ascontiguousarray(a["t1"][np.ix_(po, pv)]),
                t2=np.ascontiguousarray(a["t2"][np.ix_(po, po, pv, pv)]))


def need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_18553_gb300 as te
    from paper_2412_18553_gb300.build import build
    build()
    return te
