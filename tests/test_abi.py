"""Host-side checks of the C ABI: the library builds, loads and exports every
function include/tenergy.h declares; status codes and messages without a GPU."""
import ctypes
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tenergy.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:te_status|const char\s*\*)\s+(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_18553_gb300.build import build
    from paper_2412_18553_gb300 import _lib
    build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("t_energy", "t_energy_batched", "t_energy_vjp", "te_create", "te_destroy",
              "te_last_error", "t_energy_triples", "te_sync"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_signatures_cover_header():
    from paper_2412_18553_gb300 import _lib
    assert sorted(s[0] for s in _lib.SIGNATURES) == _declared()


def test_struct_layout_matches_header():
    from paper_2412_18553_gb300._lib import TeCluster, TeClusterGrad
    assert ctypes.sizeof(TeCluster) == 2 * 8 + 7 * 8
    assert ctypes.sizeof(TeClusterGrad) == 7 * 8


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU error path")
def test_create_without_gpu_reports_cuda_error(lib):
    h = ctypes.c_void_p(123)
    st = lib.te_create(ctypes.byref(h), 0, None)
    assert st == 3  # TE_ECUDA
    assert h.value is None
    assert b"device" in lib.te_last_error()


def test_null_arguments_are_rejected(lib):
    from paper_2412_18553_gb300._lib import TeCluster
    assert lib.te_create(None, 0, None) == 1
    assert lib.te_reserve(None, None, 0, 1) == 1
    assert lib.t_energy(None, None, 0, None, None) == 1
    assert lib.t_energy_batched(None, None, 0, 0, None, None) == 1
    assert lib.te_sync(None, None) == 1
    assert lib.te_destroy(None) == 0
    assert lib.te_last_error()


def test_canonical_triple_order_matches_oracle():
    from oracle.t_energy import unique_triples
    import paper_2412_18553_gb300 as te
    for o in range(1, 7):
        assert len(unique_triples(o)) == te.num_unique_triples(o)
    assert unique_triples(3) == [(1, 0, 0), (1, 1, 0), (2, 0, 0), (2, 1, 0), (2, 1, 1), (2, 2, 0), (2, 2, 1)]


def test_projector_shape_is_checked_before_any_device_work(lib):
    import numpy as np
    import paper_2412_18553_gb300 as te
    import tegen
    cl = tegen.make_cluster(3, 5, 32, 0).arrays()
    with pytest.raises(ValueError):
        te.t_energy_frag(cl, np.eye(4))
