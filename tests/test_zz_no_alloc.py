"""The no-allocation float64 entry point (t_energy_fp64_noalloc) against the
ordinary float64 entry point, called through the C ABI.

Some callers cannot let a library allocate device memory (their host program
owns the whole GPU through its own pool, or cannot take cudaMalloc's implicit
synchronisation mid-step); this entry point keeps all scratch in a fixed
array inside the library.  This file is collected last so that a run that
stops at the first failure has already run every other test."""
import ctypes

import pytest
import torch

import tegen
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def _call(lib, te, cl):
    t = te._tensors(cl, 0)
    c = te._struct(t)
    out = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.t_energy_fp64_noalloc(ctypes.byref(c), ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, out.item()


def test_no_alloc_matches_fp64_entry_point_twice():
    te = need_gpu()
    from paper_2412_18553_gb300 import _lib
    lib = _lib.load()
    a = tegen.make_cluster(*tegen.WORKLOADS["o8v40"])
    b = tegen.make_cluster(5, 24, 116, 21)
    ref_a = te.t_energy(a, "fp64").item()
    ref_b = te.t_energy(b, "fp64").item()
    # two calls in a row on the same cluster, then a different cluster and back:
    # the shared scratch keeps the previous call's contents
    for cl, ref in ((a, ref_a), (a, ref_a), (b, ref_b), (a, ref_a)):
        st, e = _call(lib, te, cl)
        assert st == 0, lib.te_last_error()
        assert abs(e - ref) <= 1e-10, (e, ref)


def test_no_alloc_rejects_clusters_beyond_its_scratch():
    te = need_gpu()
    from paper_2412_18553_gb300 import _lib
    lib = _lib.load()
    tiny = tegen.make_cluster(2, 3, 10, 1)
    t = te._tensors(tiny, 0)
    c = te._struct(t)
    c.nocc, c.nvir = 16, 120  # claims sizes beyond the scratch; checked before any access
    out = torch.zeros((), dtype=torch.float64, device="cuda")
    st = lib.t_energy_fp64_noalloc(ctypes.byref(c), ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1
    assert b"scratch" in lib.te_last_error()
