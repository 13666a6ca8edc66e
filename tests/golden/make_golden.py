"""Write oracle expected values for the GPU parity tests.

Calls only ``oracle`` and the input generator ``tegen``.  For each named
single-cluster workload it stores E(T) and the per-triple shares in canonical
triple order, plus checksums of the generated inputs so a test can detect a
generator that drew different numbers.

    python tests/golden/make_golden.py o8v40 o16v120 o32v320:sample o16v120:frag \
        o16v120:grad v8o:grad
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


# Gradient samples (the adjoint's parity at the gradient workload): the
# oracle's reverse-mode gradient over every unique triple, at 64 seeded entries
# of each input (all entries when fewer) plus each tensor's largest entry,
# with each tensor's largest magnitude (the scale of the relative bar).
GRAD_SAMPLE = 64
GRAD_BATCH_MEMBERS = {"v8o": [11, 14]}  # the smallest members of the 16-cluster v = 8 nocc batch


def grad_record(cl, label, rng_seed):
    c = O.inputs(**cl.arrays())
    t = time.time()
    e, g = O.t_energy_grad(c)
    rng = np.random.default_rng(rng_seed)
    ent = {}
    for n in O.NAMES:
        a = g[n].numpy().ravel()
        k = min(GRAD_SAMPLE, a.size)
        idx = set(int(i) for i in rng.choice(a.size, k, replace=False))
        idx.add(int(np.argmax(np.abs(a))))
        idx = sorted(idx)
        ent[n] = dict(index=idx, value=[float(a[i]) for i in idx], max_abs=float(np.max(np.abs(a))),
                      shape=list(g[n].shape))
    print(label, "E", e, f"{time.time() - t:.1f}s", flush=True)
    return dict(e_t=float(e), grad=ent, checksums=checksums(cl), oracle_seconds=time.time() - t)


def main_grad(name):
    if name in GRAD_BATCH_MEMBERS:
        members = []
        for s in GRAD_BATCH_MEMBERS[name]:
            o, v, naux, rng = tegen.batch_sizes(s, name)
            cl = tegen.make_cluster(o, v, naux, s, rng=rng)
            rec = grad_record(cl, f"{name} seed {s}", 1000 + s)
            rec.update(seed=s, nocc=o, nvir=v, naux=naux)
            members.append(rec)
        out = dict(batch=name, members=members)
    else:
        o, v, naux, seed = tegen.WORKLOADS[name]
        cl = tegen.make_cluster(o, v, naux, seed)
        out = grad_record(cl, name, 1000 + seed)
        out.update(workload=name, nocc=o, nvir=v, naux=naux, seed=seed)
    with open(os.path.join(HERE, f"oracle_{name}_grad.json"), "w") as f:
        json.dump(out, f)


def main(names):
    torch.set_num_threads(os.cpu_count() or 1)
    for name in names:
        if name.endswith(":sample"):
            main_sample(name.split(":")[0])
            continue
        if name.endswith(":grad"):
            main_grad(name.split(":")[0])
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
