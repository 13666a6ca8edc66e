"""Write oracle expected values for the GPU parity tests.

Calls only ``oracle`` and the input generator ``tegen``.  For each named
single-cluster workload it stores E(T) and the per-triple shares in canonical
triple order, plus checksums of the generated inputs so a test can detect a
generator that drew different numbers.

    python tests/golden/make_golden.py o8v40 o16v120
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import tegen  # noqa: E402
from oracle import t_energy as O  # noqa: E402


def checksums(cl):
    return {n: [float(np.sum(a)), float(np.sum(np.abs(a)))] for n, a in cl.arrays().items()}


def main(names):
    torch.set_num_threads(os.cpu_count() or 1)
    for name in names:
        o, v, naux, seed = tegen.WORKLOADS[name]
        cl = tegen.make_cluster(o, v, naux, seed)
        c = O.inputs(**cl.arrays())
        t = time.time()
        shares = [float(O.triple_share(c, i, j, k)) for (i, j, k) in O.unique_triples(o)]
        e = float(sum(shares))
        out = dict(workload=name, nocc=o, nvir=v, naux=naux, seed=seed, e_t=e,
                   shares=shares, checksums=checksums(cl), oracle_seconds=time.time() - t)
        with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as f:
            json.dump(out, f)
        print(name, e, f"{time.time() - t:.1f}s")


if __name__ == "__main__":
    main(sys.argv[1:] or ["o8v40"])
