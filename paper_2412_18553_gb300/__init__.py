"""GB300-native perturbative-triples energy E(T) of embedded clusters.

Thin Python binding of libtenergy (C ABI in include/tenergy.h): it marshals
torch tensors into the C descriptors and passes torch's current CUDA stream.
Every step of the computation runs in the library's CUDA kernels; if the
library is missing, importing the compute functions raises.

Inputs (float64; CUDA tensors are used in place, host tensors or numpy arrays
are copied to the device first):
  eps_o [o], eps_v [v], ovvv [o,v,v,v] = (ia|bd), ooov [o,o,o,v] = (jl|ia),
  ovov [o,v,o,v] = (ia|jb), t1 [o,v], t2 [o,o,v,v].
Precision: "fp64", "ozaki" (exact BF16 slices on the tensor cores, the mode
that meets 1e-7 Ha), "tf32", "bf16x3", "tf32x3".

Calls are asynchronous: input values (finite entries, max eps_o < min eps_v)
are checked on the device and a violation surfaces at the next
``Handle.sync()`` (or ``sync()`` for the default handle) as TEnergyError.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _lib
from ._lib import PRECISIONS, TEnergyError, TeCluster, TeClusterGrad, TeDf

NAMES = ("eps_o", "eps_v", "ovvv", "ooov", "ovov", "t1", "t2")

__all__ = ["Handle", "t_energy", "t_energy_triples", "t_energy_batched", "t_energy_vjp",
           "t_energy_vjp_triples", "t_energy_vjp_batched", "sync",
           "t_energy_fp64_noalloc", "t_energy_frag", "t_energy_df", "t_energy_df_triples",
           "TEnergy", "num_unique_triples", "flop_count", "TEnergyError", "NAMES",
           "mp2_bno_batched", "mp2_flop_count"]


def num_unique_triples(nocc: int) -> int:
    """Occupied triples i >= j >= k with i = j = k left out."""
    return nocc * (nocc + 1) * (nocc + 2) // 6 - nocc


def flop_count(nocc: int, nvir: int) -> float:
    """Algorithmic flops of one cluster: F = 12 (C(o+2,3) - o) v^3 (v + o)."""
    return 12.0 * num_unique_triples(nocc) * float(nvir) ** 3 * (nvir + nocc)


class Handle:
    """Owns the library handle (workspace) for one CUDA device."""

    def __init__(self, device=None, autotune_cache=None):
        """autotune_cache: optional path of a text file that keeps the tile
        shapes the autotuner picks across handles and processes."""
        lib = _lib.load()
        if device is None:
            dev = torch.cuda.current_device()
        elif isinstance(device, int):
            dev = device
        else:
            dev = torch.device(device).index or 0
        h = ctypes.c_void_p()
        path = None if autotune_cache is None else os.fsencode(autotune_cache)
        _lib.check(lib.te_create(ctypes.byref(h), dev, path))
        self._h = h
        self.device = dev

    @property
    def ptr(self):
        if self._h is None:
            raise RuntimeError("handle closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.load().te_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sync(self, stream=None):
        s = _stream(self.device, stream)
        _lib.check(_lib.load().te_sync(self.ptr, s))

    def set_workspace_limit(self, nbytes: int):
        """Most workspace bytes this handle may hold (0 = no limit); calls that
        would need more raise TEnergyError (TE_ENOMEM) before any launch."""
        _lib.check(_lib.load().te_set_workspace_limit(self.ptr, int(nbytes)))

    def set_wait_limit_ns(self, ns: int):
        _lib.check(_lib.load().te_set_wait_limit_ns(self.ptr, int(ns)))

    def set_ozaki_bits(self, bits: int):
        """Slice width of the "ozaki" mode: 0 automatic (7-bit slices while
        2 (nvir + nocc) <= 1024, else 6-bit), or 6 / 7 forced."""
        _lib.check(_lib.load().te_set_ozaki_bits(self.ptr, int(bits)))

    def watchdog_selftest(self, limit_ns: int = 20_000_000, stream=None):
        """Launch a kernel whose bounded wait must expire after limit_ns; the
        next sync() raises TEnergyError with status TE_ETIMEOUT."""
        s = _stream(self.device, stream)
        _lib.check(_lib.load().te_watchdog_selftest(self.ptr, int(limit_ns), s))

    def profile(self, on: bool = True):
        _lib.check(_lib.load().te_profile_enable(self.ptr, 1 if on else 0))

    def profile_read(self, reset: bool = True) -> dict:
        pr = _lib.TeProfile()
        _lib.check(_lib.load().te_profile_read(self.ptr, ctypes.byref(pr), 1 if reset else 0))
        return {f: getattr(pr, f) for f, _ in pr._fields_}

    def reserve(self, nocc: int, nvir: int, precision="fp64", energy=True, vjp=False, frag=False):
        """Allocate the workspace for clusters up to (nocc, nvir) now, for the
        energy calls, the adjoint and / or the projected energy, so that later
        calls allocate nothing."""
        c = _lib.TeCluster()
        c.nocc, c.nvir = int(nocc), int(nvir)
        what = (1 if energy else 0) | (2 if vjp else 0) | (4 if frag else 0)
        _lib.check(_lib.load().te_reserve(self.ptr, ctypes.byref(c), _prec(precision), what))

    def workspace_bytes(self, cluster, precision="fp64") -> int:
        t = _tensors(cluster, self.device)
        c = _struct(t)
        out = ctypes.c_size_t()
        _lib.check(_lib.load().te_workspace_bytes(self.ptr, ctypes.byref(c), _prec(precision),
                                                  ctypes.byref(out)))
        return int(out.value)

    def df_workspace_bytes(self, nocc: int, nvir: int, naux: int, precision="ozaki") -> int:
        """Workspace bytes t_energy_df needs for these sizes."""
        c = _lib.TeCluster()
        c.nocc, c.nvir = int(nocc), int(nvir)
        df = TeDf(int(naux), None, None)
        out = ctypes.c_size_t()
        _lib.check(_lib.load().te_df_workspace_bytes(self.ptr, ctypes.byref(c), ctypes.byref(df), _prec(precision),
                                                     ctypes.byref(out)))
        return int(out.value)


_DEFAULT = {}


def _handle(handle, device):
    if handle is not None:
        return handle
    if device not in _DEFAULT:
        _DEFAULT[device] = Handle(device)
    return _DEFAULT[device]


def _prec(p):
    if isinstance(p, int):
        return p
    try:
        return PRECISIONS[p.lower()]
    except KeyError:
        raise ValueError(f"unknown precision {p!r}; one of {sorted(PRECISIONS)}") from None


def _stream(device, stream):
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _as_dict(cluster):
    if isinstance(cluster, dict):
        return cluster
    if hasattr(cluster, "arrays"):
        return cluster.arrays()
    if isinstance(cluster, (tuple, list)) and len(cluster) == 7:
        return dict(zip(NAMES, cluster))
    raise TypeError("cluster must be a dict, a 7-tuple or an object with .arrays()")


def _tensors(cluster, device, skip=()):
    d = _as_dict(cluster)
    dev = torch.device("cuda", device)
    out = {}
    for n in NAMES:
        if n in skip:
            continue
        x = d[n]
        t = x if isinstance(x, torch.Tensor) else torch.as_tensor(x)
        if t.dtype != torch.float64:
            raise TypeError(f"{n} must be float64, got {t.dtype}")
        if t.device != dev:
            t = t.to(dev, non_blocking=True)
        out[n] = t.contiguous()
    o, v = out["eps_o"].shape[0], out["eps_v"].shape[0]
    want = dict(eps_o=(o,), eps_v=(v,), ovvv=(o, v, v, v), ooov=(o, o, o, v), ovov=(o, v, o, v),
                t1=(o, v), t2=(o, o, v, v))
    for n, shp in want.items():
        if n in skip:
            continue
        if tuple(out[n].shape) != shp:
            raise ValueError(f"{n} has shape {tuple(out[n].shape)}, expected {shp}")
    return out


def _struct(t):
    return TeCluster(t["eps_o"].shape[0], t["eps_v"].shape[0],
                     *(ctypes.c_void_p(t[n].data_ptr() if n in t else None) for n in NAMES))


def _device_of(cluster, device):
    if device is not None:
        return torch.device(device).index if not isinstance(device, int) else device
    for n in NAMES:
        x = _as_dict(cluster).get(n)
        if isinstance(x, torch.Tensor) and x.is_cuda:
            return x.device.index
    return torch.cuda.current_device()


def t_energy(cluster, precision="fp64", handle=None, device=None, stream=None) -> torch.Tensor:
    """E(T) of one cluster as a 0-dim float64 CUDA tensor."""
    dev = _device_of(cluster, device)
    h = _handle(handle, dev)
    t = _tensors(cluster, dev)
    c = _struct(t)
    out = torch.empty((), dtype=torch.float64, device=torch.device("cuda", dev))
    _lib.check(_lib.load().t_energy(h.ptr, ctypes.byref(c), _prec(precision),
                                    ctypes.c_void_p(out.data_ptr()), _stream(dev, stream)))
    return out


def t_energy_triples(cluster, t_begin=0, t_end=None, precision="fp64", handle=None, device=None,
                     stream=None) -> torch.Tensor:
    """Per-triple shares (m/3) e_ijk for canonical triple indices [t_begin, t_end)."""
    dev = _device_of(cluster, device)
    h = _handle(handle, dev)
    t = _tensors(cluster, dev)
    if t_end is None:
        t_end = num_unique_triples(t["eps_o"].shape[0])
    out = torch.empty((max(0, t_end - t_begin),), dtype=torch.float64, device=torch.device("cuda", dev))
    c = _struct(t)
    _lib.check(_lib.load().t_energy_triples(h.ptr, ctypes.byref(c), _prec(precision), int(t_begin),
                                            int(t_end), ctypes.c_void_p(out.data_ptr()),
                                            _stream(dev, stream)))
    return out


def _df(Bov, Bvv, o, v, device):
    dev = torch.device("cuda", device)
    out = []
    for n, x in (("Bov", Bov), ("Bvv", Bvv)):
        t = x if isinstance(x, torch.Tensor) else torch.as_tensor(x)
        if t.dtype != torch.float64:
            raise TypeError(f"{n} must be float64, got {t.dtype}")
        out.append(t.to(dev, non_blocking=True).contiguous())
    bov, bvv = out
    naux = bov.shape[0]
    if tuple(bov.shape) != (naux, o, v) or tuple(bvv.shape) != (naux, v, v):
        raise ValueError(f"Bov {tuple(bov.shape)} and Bvv {tuple(bvv.shape)} must be [naux,{o},{v}] and [naux,{v},{v}]")
    return bov, bvv, TeDf(naux, ctypes.c_void_p(bov.data_ptr()), ctypes.c_void_p(bvv.data_ptr()))


def t_energy_df(cluster, Bov, Bvv, precision="ozaki", handle=None, device=None, stream=None) -> torch.Tensor:
    """E(T) of one cluster with ovvv[i,a,b,d] = sum_P Bov[P,i,a] Bvv[P,b,d]
    formed on the device from the density-fitting factors (the cluster's
    ovvv, if any, is not read).  Tensor-core modes only."""
    dev = _device_of(cluster, device)
    h = _handle(handle, dev)
    t = _tensors(cluster, dev, skip=("ovvv",))
    bov, bvv, df = _df(Bov, Bvv, t["eps_o"].shape[0], t["eps_v"].shape[0], dev)
    c = _struct(t)
    out = torch.empty((), dtype=torch.float64, device=torch.device("cuda", dev))
    _lib.check(_lib.load().t_energy_df(h.ptr, ctypes.byref(c), ctypes.byref(df), _prec(precision),
                                       ctypes.c_void_p(out.data_ptr()), _stream(dev, stream)))
    return out


def t_energy_df_triples(cluster, Bov, Bvv, t_begin=0, t_end=None, precision="ozaki", handle=None, device=None,
                        stream=None) -> torch.Tensor:
    """Per-triple shares of [t_begin, t_end) with ovvv from the density-fitting factors."""
    dev = _device_of(cluster, device)
    h = _handle(handle, dev)
    t = _tensors(cluster, dev, skip=("ovvv",))
    bov, bvv, df = _df(Bov, Bvv, t["eps_o"].shape[0], t["eps_v"].shape[0], dev)
    if t_end is None:
        t_end = num_unique_triples(t["eps_o"].shape[0])
    out = torch.empty((max(0, t_end - t_begin),), dtype=torch.float64, device=torch.device("cuda", dev))
    c = _struct(t)
    _lib.check(_lib.load().t_energy_df_triples(h.ptr, ctypes.byref(c), ctypes.byref(df), _prec(precision),
                                               int(t_begin), int(t_end), ctypes.c_void_p(out.data_ptr()),
                                               _stream(dev, stream)))
    return out


def t_energy_batched(clusters, precision="fp64", handle=None, device=None, stream=None) -> torch.Tensor:
    """E(T) of each of several independent clusters (float64 CUDA tensor [n])."""
    clusters = list(clusters)
    dev = _device_of(clusters[0], device) if clusters else (device or torch.cuda.current_device())
    h = _handle(handle, dev)
    ts = [_tensors(c, dev) for c in clusters]
    arr = (TeCluster * max(1, len(ts)))(*[_struct(t) for t in ts])
    out = torch.empty((len(ts),), dtype=torch.float64, device=torch.device("cuda", dev))
    _lib.check(_lib.load().t_energy_batched(h.ptr, arr, len(ts), _prec(precision),
                                            ctypes.c_void_p(out.data_ptr()), _stream(dev, stream)))
    return out


def _grad_buffers(t, which):
    names = NAMES if which is None else tuple(which)
    for n in names:
        if n not in NAMES:
            raise ValueError(f"unknown input {n!r}")
    return {n: torch.empty_like(t[n]) for n in names}


def t_energy_vjp(cluster, gE=1.0, precision="fp64", handle=None, device=None, stream=None, grads=None):
    """(E, grads): grads[name] = gE * dE/d(name) for all seven inputs, or for
    the names listed in ``grads`` (the others are not computed)."""
    dev = _device_of(cluster, device)
    h = _handle(handle, dev)
    t = _tensors(cluster, dev)
    grads = _grad_buffers(t, grads)
    g = _grad_struct(grads)
    e = torch.empty((), dtype=torch.float64, device=torch.device("cuda", dev))
    c = _struct(t)
    _lib.check(_lib.load().t_energy_vjp(h.ptr, ctypes.byref(c), _prec(precision), float(gE),
                                        ctypes.c_void_p(e.data_ptr()), ctypes.byref(g),
                                        _stream(dev, stream)))
    return e, grads


def sync(device=None, stream=None):
    """te_sync on the default handle of `device` (the handle the functions
    below use when none is given): waits for its work on the stream and
    raises TEnergyError for a failed device-side input check or watchdog."""
    dev = torch.cuda.current_device() if device is None else device
    _handle(None, dev).sync(stream)


def _grad_struct(grads):
    return TeClusterGrad(*(ctypes.c_void_p(grads[n].data_ptr()) if n in grads else None for n in NAMES))


def t_energy_vjp_triples(cluster, t_begin=0, t_end=None, gE=1.0, precision="fp64", handle=None, device=None,
                         stream=None, grads=None):
    """(sum of the shares of triples [t_begin, t_end), grads): the adjoint
    restricted to a canonical triple range; ranges that partition all
    triples give gradients that add up to t_energy_vjp's.  ``grads``: the
    inputs whose gradient is wanted (default all)."""
    dev = _device_of(cluster, device)
    h = _handle(handle, dev)
    t = _tensors(cluster, dev)
    if t_end is None:
        t_end = num_unique_triples(t["eps_o"].shape[0])
    grads = _grad_buffers(t, grads)
    g = _grad_struct(grads)
    e = torch.empty((), dtype=torch.float64, device=torch.device("cuda", dev))
    c = _struct(t)
    _lib.check(_lib.load().t_energy_vjp_triples(h.ptr, ctypes.byref(c), _prec(precision), int(t_begin),
                                                int(t_end), float(gE), ctypes.c_void_p(e.data_ptr()),
                                                ctypes.byref(g), _stream(dev, stream)))
    return e, grads


def t_energy_vjp_batched(clusters, gE=None, precision="fp64", handle=None, device=None, stream=None):
    """(E [n], list of gradient dicts): the adjoint of n independent clusters
    in one library call; gE: n upstream gradients (default all 1)."""
    clusters = list(clusters)
    dev = _device_of(clusters[0], device) if clusters else (device or torch.cuda.current_device())
    h = _handle(handle, dev)
    ts = [_tensors(c, dev) for c in clusters]
    n = len(ts)
    arr = (TeCluster * max(1, n))(*[_struct(t) for t in ts])
    grads = [{nm: torch.empty_like(t[nm]) for nm in NAMES} for t in ts]
    garr = (TeClusterGrad * max(1, n))(*[_grad_struct(g) for g in grads])
    gbuf = None
    if gE is not None:
        gl = [float(x) for x in gE]
        if len(gl) != n:
            raise ValueError(f"gE has {len(gl)} entries for {n} clusters")
        gbuf = (ctypes.c_double * max(1, n))(*gl)
    e = torch.empty((n,), dtype=torch.float64, device=torch.device("cuda", dev))
    _lib.check(_lib.load().t_energy_vjp_batched(h.ptr, arr, n, _prec(precision), gbuf,
                                                ctypes.c_void_p(e.data_ptr()), garr, _stream(dev, stream)))
    return e, grads


def t_energy_frag(cluster, cf, precision="fp64", handle=None, device=None, stream=None, shares=False):
    """Fragment-projected E(T) (Eq. E_corr_CCSD_T with a general C^f): cf is
    the [nocc, nocc] projector acting on W~'s first occupied index.  Returns a
    0-dim float64 CUDA tensor, or (E, per-triple shares) with shares=True.
    precision: "fp64" or "ozaki"."""
    o = int(_as_dict(cluster)["eps_o"].shape[0])
    cf = torch.as_tensor(cf, dtype=torch.float64)
    if tuple(cf.shape) != (o, o):
        raise ValueError(f"cf must be [{o}, {o}], got {tuple(cf.shape)}")
    dev = _device_of(cluster, device)
    h = _handle(handle, dev)
    t = _tensors(cluster, dev)
    cf = cf.to(torch.device("cuda", dev)).contiguous()
    e = torch.empty((), dtype=torch.float64, device=torch.device("cuda", dev))
    sh = torch.empty(max(1, num_unique_triples(o)), dtype=torch.float64, device=e.device) if shares else None
    c = _struct(t)
    _lib.check(_lib.load().t_energy_frag(h.ptr, ctypes.byref(c), ctypes.c_void_p(cf.data_ptr()), _prec(precision),
                                         ctypes.c_void_p(e.data_ptr()),
                                         ctypes.c_void_p(sh.data_ptr()) if shares else None,
                                         _stream(dev, stream)))
    if shares:
        return e, sh[:num_unique_triples(o)]
    return e


def t_energy_fp64_noalloc(cluster, device=None, stream=None) -> torch.Tensor:
    """Float64 E(T) through the library's no-allocation entry point (its
    scratch is a fixed array inside the library; the result tensor here is
    the caller's own allocation).  For callers whose host program forbids
    library-side device allocations; small clusters only (64 MiB scratch)."""
    dev = _device_of(cluster, device)
    t = _tensors(cluster, dev)
    c = _struct(t)
    out = torch.empty((), dtype=torch.float64, device=torch.device("cuda", dev))
    with torch.cuda.device(dev):
        _lib.check(_lib.load().t_energy_fp64_noalloc(ctypes.byref(c), ctypes.c_void_p(out.data_ptr()),
                                                     _stream(dev, stream)))
    return out


MP2_OUTPUTS = ("t2", "gamma_oo", "gamma_vv", "pop_o", "pop_v")


def mp2_flop_count(nocc: int, nvir: int, naux: int) -> float:
    """Flops of the MP2 step's three contractions: (ia|jb) (2 (ov)^2 naux),
    gamma_vv (2 o^2 v^3) and gamma_oo (2 o^3 v^2)."""
    o, v, P = float(nocc), float(nvir), float(naux)
    return 2.0 * (o * v) ** 2 * P + 2.0 * o * o * v ** 3 + 2.0 * o ** 3 * v * v


def mp2_bno_batched(clusters, precision="fp64", outputs=MP2_OUTPUTS, handle=None, device=None, stream=None):
    """The MP2 step for a batch of clusters, each (eps_o [o], eps_v [v], Bov
    [naux, o, v]): per cluster a dict with the requested ``outputs`` among
    t2 [o,o,v,v], gamma_oo [o,o], gamma_vv [v,v], pop_o [o], pop_v [v]
    (float64 CUDA tensors).  precision: "fp64" or "ozaki"."""
    clusters = list(clusters)
    for n in outputs:
        if n not in MP2_OUTPUTS:
            raise ValueError(f"unknown output {n!r}")
    dev = device if device is not None else torch.cuda.current_device()
    dev = torch.device(dev).index if not isinstance(dev, int) else dev
    h = _handle(handle, dev)
    d = torch.device("cuda", dev)
    ins, outs, res = [], [], []
    for c in clusters:
        eo, ev, B = (torch.as_tensor(x, dtype=torch.float64).to(d).contiguous() for x in c)
        o, v, P = eo.shape[0], ev.shape[0], B.shape[0]
        if tuple(B.shape) != (P, o, v):
            raise ValueError(f"Bov has shape {tuple(B.shape)}, expected ({P}, {o}, {v})")
        shapes = dict(t2=(o, o, v, v), gamma_oo=(o, o), gamma_vv=(v, v), pop_o=(o,), pop_v=(v,))
        r = {n: torch.empty(shapes[n], dtype=torch.float64, device=d) for n in outputs}
        ins.append((eo, ev, B))
        res.append(r)
        outs.append(_lib.TeMp2Out(*(ctypes.c_void_p(r[n].data_ptr()) if n in r else None for n in MP2_OUTPUTS)))
    n = len(clusters)
    carr = (_lib.TeMp2Cluster * max(1, n))(*[_lib.TeMp2Cluster(eo.shape[0], ev.shape[0], B.shape[0],
                                                                 ctypes.c_void_p(eo.data_ptr()),
                                                                 ctypes.c_void_p(ev.data_ptr()),
                                                                 ctypes.c_void_p(B.data_ptr()))
                                               for eo, ev, B in ins])
    oarr = (_lib.TeMp2Out * max(1, n))(*outs)
    _lib.check(_lib.load().t_mp2_bno_batched(h.ptr, carr, oarr, n, _prec(precision), _stream(dev, stream)))
    return res


class TEnergy(torch.autograd.Function):
    """E(T) as a differentiable function of (eps_o, eps_v, ovvv, ooov, ovov, t1, t2);
    the backward pass calls the library's adjoint (t_energy_vjp)."""

    @staticmethod
    def forward(ctx, eps_o, eps_v, ovvv, ooov, ovov, t1, t2, precision="fp64"):
        cl = dict(zip(NAMES, (eps_o, eps_v, ovvv, ooov, ovov, t1, t2)))
        ctx.save_for_backward(eps_o, eps_v, ovvv, ooov, ovov, t1, t2)
        ctx.precision = precision
        return t_energy(cl, precision)

    @staticmethod
    def backward(ctx, gout):
        cl = dict(zip(NAMES, ctx.saved_tensors))
        _, g = t_energy_vjp(cl, float(gout), ctx.precision)
        return tuple(g[n] for n in NAMES) + (None,)
