"""ctypes declarations of the C ABI in include/tenergy.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from .build import LIB

c_int64 = ctypes.c_int64
c_void_p = ctypes.c_void_p

TE_OK, TE_EINVAL, TE_ENOMEM, TE_ECUDA, TE_ETIMEOUT, TE_EUNSUPPORTED = range(6)
STATUS_NAMES = {0: "TE_OK", 1: "TE_EINVAL", 2: "TE_ENOMEM", 3: "TE_ECUDA",
                4: "TE_ETIMEOUT", 5: "TE_EUNSUPPORTED"}
PRECISIONS = {"fp64": 0, "tf32": 1, "bf16x3": 2, "tf32x3": 3, "ozaki": 4}


class TeCluster(ctypes.Structure):
    _fields_ = [("nocc", c_int64), ("nvir", c_int64),
                ("eps_o", c_void_p), ("eps_v", c_void_p), ("ovvv", c_void_p),
                ("ooov", c_void_p), ("ovov", c_void_p), ("t1", c_void_p), ("t2", c_void_p)]


class TeClusterGrad(ctypes.Structure):
    _fields_ = [("eps_o", c_void_p), ("eps_v", c_void_p), ("ovvv", c_void_p),
                ("ooov", c_void_p), ("ovov", c_void_p), ("t1", c_void_p), ("t2", c_void_p)]


class TeMp2Cluster(ctypes.Structure):
    _fields_ = [("nocc", c_int64), ("nvir", c_int64), ("naux", c_int64),
                ("eps_o", c_void_p), ("eps_v", c_void_p), ("Bov", c_void_p)]


class TeMp2Out(ctypes.Structure):
    _fields_ = [("t2", c_void_p), ("gamma_oo", c_void_p), ("gamma_vv", c_void_p),
                ("pop_o", c_void_p), ("pop_v", c_void_p)]


class TeDf(ctypes.Structure):
    _fields_ = [("naux", c_int64), ("Bov", c_void_p), ("Bvv", c_void_p)]


class TeProfile(ctypes.Structure):
    _fields_ = [("launches", c_int64), ("gemm_launches", c_int64), ("gemm_ms", ctypes.c_double),
                ("energy_launches", c_int64), ("energy_ms", ctypes.c_double),
                ("gemm_flops", ctypes.c_double)]


# (name, restype, argtypes) for every function of include/tenergy.h
SIGNATURES = [
    ("te_create", ctypes.c_int, [ctypes.POINTER(c_void_p), ctypes.c_int, ctypes.c_char_p]),
    ("te_reserve", ctypes.c_int, [c_void_p, ctypes.POINTER(TeCluster), ctypes.c_int, ctypes.c_int]),
    ("te_destroy", ctypes.c_int, [c_void_p]),
    ("t_energy", ctypes.c_int, [c_void_p, ctypes.POINTER(TeCluster), ctypes.c_int, c_void_p, c_void_p]),
    ("t_energy_triples", ctypes.c_int, [c_void_p, ctypes.POINTER(TeCluster), ctypes.c_int,
                                        c_int64, c_int64, c_void_p, c_void_p]),
    ("t_energy_batched", ctypes.c_int, [c_void_p, ctypes.POINTER(TeCluster), c_int64, ctypes.c_int,
                                        c_void_p, c_void_p]),
    ("t_energy_vjp", ctypes.c_int, [c_void_p, ctypes.POINTER(TeCluster), ctypes.c_int, ctypes.c_double,
                                    c_void_p, ctypes.POINTER(TeClusterGrad), c_void_p]),
    ("t_energy_vjp_triples", ctypes.c_int, [c_void_p, ctypes.POINTER(TeCluster), ctypes.c_int, c_int64, c_int64,
                                            ctypes.c_double, c_void_p, ctypes.POINTER(TeClusterGrad), c_void_p]),
    ("t_energy_vjp_batched", ctypes.c_int, [c_void_p, ctypes.POINTER(TeCluster), c_int64, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_double), c_void_p,
                                            ctypes.POINTER(TeClusterGrad), c_void_p]),
    ("t_energy_frag", ctypes.c_int, [c_void_p, ctypes.POINTER(TeCluster), c_void_p, ctypes.c_int,
                                     c_void_p, c_void_p, c_void_p]),
    ("t_energy_df", ctypes.c_int, [c_void_p, ctypes.POINTER(TeCluster), ctypes.POINTER(TeDf), ctypes.c_int,
                                   c_void_p, c_void_p]),
    ("t_energy_df_triples", ctypes.c_int, [c_void_p, ctypes.POINTER(TeCluster), ctypes.POINTER(TeDf), ctypes.c_int,
                                           c_int64, c_int64, c_void_p, c_void_p]),
    ("te_df_workspace_bytes", ctypes.c_int, [c_void_p, ctypes.POINTER(TeCluster), ctypes.POINTER(TeDf),
                                             ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    ("te_sync", ctypes.c_int, [c_void_p, c_void_p]),
    ("te_workspace_bytes", ctypes.c_int, [c_void_p, ctypes.POINTER(TeCluster), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_size_t)]),
    ("te_last_error", ctypes.c_char_p, []),
    ("te_set_wait_limit_ns", ctypes.c_int, [c_void_p, ctypes.c_uint64]),
    ("te_set_workspace_limit", ctypes.c_int, [c_void_p, ctypes.c_size_t]),
    ("te_watchdog_selftest", ctypes.c_int, [c_void_p, ctypes.c_uint64, c_void_p]),
    ("te_set_ozaki_bits", ctypes.c_int, [c_void_p, ctypes.c_int]),
    ("te_profile_enable", ctypes.c_int, [c_void_p, ctypes.c_int]),
    ("te_profile_read", ctypes.c_int, [c_void_p, ctypes.POINTER(TeProfile), ctypes.c_int]),
    ("t_energy_fp64_noalloc", ctypes.c_int, [ctypes.POINTER(TeCluster), c_void_p, c_void_p]),
    ("t_mp2_bno_batched", ctypes.c_int, [c_void_p, ctypes.POINTER(TeMp2Cluster), ctypes.POINTER(TeMp2Out), c_int64,
                                         ctypes.c_int, c_void_p]),
]

_lib = None


def load(path: str = LIB):
    """Load libtenergy.so.  Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"libtenergy.so not found at {path}; build it first with "
            "`python -c 'import __graft_entry__ as g; g.build()'` "
            "(or paper_2412_18553_gb300.build.build())")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class TEnergyError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status):
    if status != TE_OK:
        msg = load().te_last_error()
        raise TEnergyError(status, msg.decode() if msg else "")
    return status
