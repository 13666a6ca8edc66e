"""Write oracle expected values for the GPU parity tests.

Calls only ``oracle`` and the input generator ``tegen``.  For each named
single-cluster workload it stores E(T) and the per-triple shares in canonical
triple order, plus checksums of the generated inputs so a test can detect a
generator that drew different numbers.

    python tests/golden/make_golden.py o8v40 o16v120 o32v320:sample o16v120:frag
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


# Workloads too large for the whole oracle: a fixed sample of canonical triple
# indices (the lightest, a middle one and the heaviest few).
SAMPLES = {"o32v320": [0, 2976, 5943, 5948, 5950, 5951]}


def main_sample(name):
    o, v, naux, seed = tegen.WORKLOADS[name]
    cl = tegen.make_cluster(o, v, naux, seed)
    c = O.inputs(**cl.arrays())
    trip = O.unique_triples(o)
    t = time.time()
    idx = SAMPLES[name]
    shares = [float(O.triple_share(c, *trip[i])) for i in idx]
    out = dict(workload=name, nocc=o, nvir=v, naux=naux, seed=seed, triple_index=idx,
               triples=[list(trip[i]) for i in idx], shares=shares, checksums=checksums(cl),
               oracle_seconds=time.time() - t)
    with open(os.path.join(HERE, f"oracle_{name}_sample.json"), "w") as f:
        json.dump(out, f)
    print(name, "sample", shares, f"{time.time() - t:.1f}s")


# Fragment-projected energy (Eq. E_corr_CCSD_T with a general C^f): a rank-6
# projector from a seeded orthogonal matrix (stored in the file, so the test
# does not depend on the machine's QR) and a sample of canonical triples.
FRAG = {"o16v120": dict(rank=6, seed=16, triple_index=[0, 1, 399, 798, 799])}


def main_frag(name):
    o, v, naux, seed = tegen.WORKLOADS[name]
    spec = FRAG[name]
    cl = tegen.make_cluster(o, v, naux, seed)
    c = O.inputs(**cl.arrays())
    u, _ = np.linalg.qr(np.random.default_rng(spec["seed"]).standard_normal((o, o)))
    cf = u[:, :spec["rank"]] @ u[:, :spec["rank"]].T
    trip = O.unique_triples(o)
    t = time.time()
    shares = []
    for i in spec["triple_index"]:
        shares.append(float(O.triple_share_projected(c, cf, *trip[i])))
        print(name, "frag triple", i, trip[i], shares[-1], f"{time.time() - t:.1f}s", flush=True)
    out = dict(workload=name, nocc=o, nvir=v, naux=naux, seed=seed, cf=cf.tolist(),
               triple_index=spec["triple_index"], triples=[list(trip[i]) for i in spec["triple_index"]],
               shares=shares, checksums=checksums(cl), oracle_seconds=time.time() - t)
    with open(os.path.join(HERE, f"oracle_{name}_frag.json"), "w") as f:
        json.dump(out, f)


def main(names):
    torch.set_num_threads(os.cpu_count() or 1)
    for name in names:
        if name.endswith(":sample"):
            main_sample(name.split(":")[0])
            continue
        if name.endswith(":frag"):
            main_frag(name.split(":")[0])
            continue
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
