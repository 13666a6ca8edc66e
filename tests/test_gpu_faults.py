"""Failure handling through the C ABI, without any GPU fault:

* input values are checked on the device by every call's first kernel: a
  non-finite entry in any of the seven arrays, or max(eps_o) >= min(eps_v),
  is reported by the next te_sync as TE_EINVAL naming the array (or the
  ordering) and the cluster, and the handle keeps working afterwards;
* a workspace budget (te_set_workspace_limit) turns a call that needs more
  into TE_ENOMEM before any launch; a real allocation failure (a workspace
  larger than the device) gives TE_ENOMEM too;
* no call synchronises its stream: after te_reserve, t_energy is captured in
  a CUDA graph and the replay gives the eager result."""
import numpy as np
import pytest
import torch

import tegen
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

NAMES = ("eps_o", "eps_v", "ovvv", "ooov", "ovov", "t1", "t2")
TE_EINVAL, TE_ENOMEM = 1, 2


@pytest.fixture(scope="module")
def te():
    return need_gpu()


def dev(arrs):
    return {n: torch.as_tensor(np.ascontiguousarray(arrs[n])).cuda() for n in NAMES}


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_entry_is_reported_at_sync(te, prec, name, bad):
    h = te.Handle(0)
    a = dev(tegen.make_cluster(3, 11, 56, 1).arrays())
    flat = a[name].view(-1)
    flat[flat.numel() // 2] = bad
    te.t_energy(a, prec, handle=h)  # returns without waiting for the device
    with pytest.raises(te.TEnergyError) as ei:
        h.sync()
    assert ei.value.status == TE_EINVAL
    assert name in str(ei.value) and "cluster 0" in str(ei.value)
    h.sync()  # the word was cleared
    good = dev(tegen.make_cluster(3, 11, 56, 1).arrays())
    e = float(te.t_energy(good, prec, handle=h))
    h.sync()
    assert np.isfinite(e) and e < 0.0


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_orbital_energy_ordering_is_reported_at_sync(te, prec):
    h = te.Handle(0)
    a = dev(tegen.make_cluster(3, 8, 40, 1).arrays())
    a["eps_o"][1] = a["eps_v"].min() + 0.1
    te.t_energy(a, prec, handle=h)
    with pytest.raises(te.TEnergyError) as ei:
        h.sync()
    assert ei.value.status == TE_EINVAL and "eps_o" in str(ei.value) and "eps_v" in str(ei.value)


def test_batched_member_is_named(te):
    h = te.Handle(0)
    cls = [dev(tegen.make_cluster(3, 9 + x, 48, x).arrays()) for x in range(3)]
    cls[2]["t2"].view(-1)[5] = float("nan")
    te.t_energy_batched(cls, "ozaki", handle=h)
    with pytest.raises(te.TEnergyError) as ei:
        h.sync()
    assert ei.value.status == TE_EINVAL and "cluster 2" in str(ei.value) and "t2" in str(ei.value)
    # the graph checks its members on every replay: fix the value, replay, no error
    cls[2]["t2"].view(-1)[5] = 0.0
    e = te.t_energy_batched(cls, "ozaki", handle=h)
    h.sync()
    assert bool(torch.isfinite(e).all())


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_adjoint_checks_inputs(te, prec):
    h = te.Handle(0)
    a = dev(tegen.make_cluster(3, 10, 52, 2).arrays())
    a["ovvv"].view(-1)[7] = float("-inf")
    te.t_energy_vjp(a, precision=prec, handle=h)
    with pytest.raises(te.TEnergyError) as ei:
        h.sync()
    assert ei.value.status == TE_EINVAL and "ovvv" in str(ei.value)


def test_workspace_limit_gives_enomem_before_any_launch(te):
    h = te.Handle(0)
    a = dev(tegen.make_cluster(4, 24, 112, 3).arrays())
    need = h.workspace_bytes(a, "ozaki")
    h.set_workspace_limit(need // 2)
    h.profile_read(reset=True)
    with pytest.raises(te.TEnergyError) as ei:
        te.t_energy(a, "ozaki", handle=h)
    assert ei.value.status == TE_ENOMEM and "limit" in str(ei.value)
    # only the input check was launched; nothing allocated or computed
    assert h.profile_read(reset=True)["gemm_launches"] == 0
    h.sync()
    h.set_workspace_limit(0)
    e = float(te.t_energy(a, "ozaki", handle=h))
    h.sync()
    assert np.isfinite(e)
    with pytest.raises(te.TEnergyError):  # below what the handle already holds
        h.set_workspace_limit(1024)


def test_allocation_failure_gives_enomem(te):
    """A workspace larger than the device: cudaMalloc fails (no fault) and the
    reservation reports TE_ENOMEM; the handle keeps working."""
    h = te.Handle(0)
    with pytest.raises(te.TEnergyError) as ei:
        h.reserve(1024, 4096, "fp64", energy=True)
    assert ei.value.status == TE_ENOMEM
    cl = tegen.make_cluster(3, 9, 48, 4)
    e = float(te.t_energy(cl, "fp64", handle=h))
    h.sync()
    assert np.isfinite(e)


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_t_energy_is_graph_capturable_after_reserve(te, prec):
    """No call synchronises or allocates once the workspace exists: the
    energy call records into a caller's CUDA graph."""
    h = te.Handle(0)
    a = dev(tegen.make_cluster(5, 40, 180, 6).arrays())
    h.reserve(5, 40, prec)
    e_eager = float(te.t_energy(a, prec, handle=h))
    h.sync()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        out = te.t_energy(a, prec, handle=h, stream=s)
    for _ in range(2):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert float(out) == e_eager
    h.sync()
