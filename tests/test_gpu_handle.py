"""Handle options through the C ABI: the autotune cache file of te_create and
the up-front workspace of te_reserve."""
import os

import numpy as np
import pytest
import torch

import tegen
from oracle import t_energy as O
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

# nvir = 64 gives the tuner three M-tile candidates; nvir = 17 gives one
SIZES = [(4, 64, 21), (3, 17, 22)]


@pytest.fixture(scope="module")
def te():
    return need_gpu()


@pytest.fixture(scope="module")
def batch():
    host = [tegen.make_cluster(o, v, 4 * (o + v), s).arrays() for o, v, s in SIZES]
    ref = [float(O.t_energy(O.inputs(**a))) for a in host]
    dev = [{n: torch.as_tensor(x).cuda() for n, x in a.items()} for a in host]
    return dev, ref


def _entries(path):
    lines = open(path).read().splitlines()
    return lines[0], [tuple(int(t) for t in ln.split()) for ln in lines[1:]]


def _header():
    p = torch.cuda.get_device_properties(0)
    return f"tenergy-autotune 1 sms={p.multi_processor_count} cc={p.major}.{p.minor}"


def _run(te, h, dev):
    h.profile_read(reset=True)
    e = te.t_energy_batched(dev, "ozaki", handle=h).cpu().numpy()
    return e, h.profile_read(reset=True)["launches"]


def test_cache_is_written_then_reused_without_tuning(te, batch, tmp_path):
    dev, ref = batch
    path = str(tmp_path / "tune.txt")
    h1 = te.Handle(0, autotune_cache=path)
    e1, n1 = _run(te, h1, dev)
    for x in range(len(ref)):
        assert abs(e1[x] - ref[x]) <= 1e-7
    head, ent = _entries(path)
    assert head == _header()
    tuned = [t for t in ent if t[:2] == (4, 64)]
    assert len(tuned) == 1 and tuned[0][3] in (16, 32, 64, 128) and tuned[0][4] >= 1
    assert not [t for t in ent if t[:2] == (3, 17)]  # one candidate: nothing to keep
    ino = os.stat(path).st_ino
    h2 = te.Handle(0, autotune_cache=path)
    e2, n2 = _run(te, h2, dev)
    assert n2 < n1  # no tuning launches
    assert os.stat(path).st_ino == ino and _entries(path)[1] == ent  # not rewritten
    np.testing.assert_allclose(e2, e1, rtol=1e-13, atol=0)


def test_other_candidate_from_the_file_is_used(te, batch, tmp_path):
    dev, ref = batch
    path = str(tmp_path / "tune.txt")
    e1, _ = _run(te, te.Handle(0, autotune_cache=path), dev)
    head, ent = _entries(path)
    (o, v, mode, tb, nnt), = [t for t in ent if t[:2] == (4, 64)]
    other = 32 if tb != 32 else 16  # both are candidates at nvir = 64
    with open(path, "w") as f:
        f.write(f"{head}\n{o} {v} {mode} {other} {nnt}\n")
    e2, _ = _run(te, te.Handle(0, autotune_cache=path), dev)
    assert _entries(path)[1] == [(o, v, mode, other, nnt)]  # kept, not retuned
    for x in range(len(ref)):
        assert abs(e2[x] - ref[x]) <= 1e-7
    np.testing.assert_allclose(e2, e1, rtol=1e-12, atol=0)


@pytest.mark.parametrize("content", [
    "tenergy-autotune 1 sms=1 cc=1.0\n4 64 {mode} 32 1\n",  # written on another GPU
    "{head}\n4 64 {mode} 8 99\nnot a line\n4 64\n",        # not a candidate, malformed
])
def test_foreign_or_bad_entries_are_ignored(te, batch, tmp_path, content):
    dev, ref = batch
    path = str(tmp_path / "tune.txt")
    _run(te, te.Handle(0, autotune_cache=path), dev)
    head, ent = _entries(path)
    mode = [t for t in ent if t[:2] == (4, 64)][0][2]
    with open(path, "w") as f:
        f.write(content.format(head=head, mode=mode))
    e, _ = _run(te, te.Handle(0, autotune_cache=path), dev)
    for x in range(len(ref)):
        assert abs(e[x] - ref[x]) <= 1e-7
    head2, ent2 = _entries(path)  # retuned and rewritten for this GPU
    assert head2 == _header()
    t = [t for t in ent2 if t[:2] == (4, 64)]
    assert len(t) == 1 and t[0][3] in (16, 32, 64, 128)


def test_unwritable_cache_path_is_not_an_error(te, batch, tmp_path):
    dev, ref = batch
    path = str(tmp_path / "no_such_dir" / "tune.txt")
    e, _ = _run(te, te.Handle(0, autotune_cache=path), dev)
    assert abs(e[0] - ref[0]) <= 1e-7
    assert not os.path.exists(path)


def test_reserve_allocates_up_front(te):
    o, v = 8, 120
    cl = tegen.make_cluster(o, v, 4 * (o + v), 5)
    a = {n: torch.as_tensor(x).cuda() for n, x in cl.arrays().items()}
    torch.cuda.synchronize()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    # without reserve the first call allocates the workspace
    h0 = te.Handle(0)
    need = h0.workspace_bytes(a, "ozaki")
    assert need > 64 << 20
    free0 = torch.cuda.mem_get_info()[0]
    te.t_energy(a, "ozaki", handle=h0)
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] >= need
    h0.close()
    # with reserve, the first energy call allocates nothing further
    h = te.Handle(0)
    h.reserve(o, v, "ozaki", energy=True, vjp=True)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    e = te.t_energy(a, "ozaki", handle=h)
    torch.cuda.synchronize()
    assert abs(free1 - torch.cuda.mem_get_info()[0]) < (4 << 20)
    e0 = te.t_energy(a, "ozaki", handle=te.Handle(0))
    assert float(e) == float(e0)
    ev, _ = te.t_energy_vjp(a, precision="ozaki", handle=h)
    assert abs(float(ev) - float(e)) <= 1e-7
    del out
    with pytest.raises(te.TEnergyError):
        h.reserve(o, v, "ozaki", energy=False, vjp=False)
    with pytest.raises(te.TEnergyError):
        h.reserve(0, v, "fp64")
