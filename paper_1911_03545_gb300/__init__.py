"""GB300 binned pair counter (Corrfunc's method, arXiv:1911.03545) -- Python binding.

The binding only marshals arguments into the C ABI of include/cf.h; every step of the count
runs in the CUDA library.  Functions carry the C names:

    ctx = cf_create(device=0, stream=torch.cuda.current_stream())
    out = cf_count(ctx, params(kind="r", edges=e, autocorr=True, periodic=True, box=L), points(x, y, z))
    cf_destroy(ctx)

Points may be torch CUDA tensors (used in place, on the context's stream) or numpy arrays
(copied by the library).  Results are numpy arrays: npairs (uint64), wsum, ravg, wp.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import _capi
from ._capi import (  # noqa: F401
    CF_DD_R, CF_DD_RPPI, CF_DD_RPPI_MOCKS, CF_DD_THETA, CF_F32, CF_F64, CF_OK, CF_OPT_AUDIT, CF_OPT_CTAS_PER_SM, CF_OPT_ITER_LIMIT,
    CF_OPT_BLOCK_PRUNE, CF_OPT_CELL_ORDER, CF_OPT_CELL_PRUNE, CF_OPT_JCHUNK, CF_OPT_MEM_CAP, CF_OPT_QUEUE, CF_OPT_REFINE, CF_OPT_THETA_GRID, CF_OPT_TILE, CF_OPT_VARIANT, CF_OPT_WARPS,
    CF_W_NONE, CF_W_PAIR_PRODUCT, CF_WP, STATUS_NAMES,
)

KINDS = {"r": CF_DD_R, "rppi": CF_DD_RPPI, "wp": CF_WP, "theta": CF_DD_THETA, "mocks": CF_DD_RPPI_MOCKS}


class CfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(rc: int, ctx=None, server=None):
    if rc != 0:
        L = _capi.lib()
        if server is not None:
            msg = L.cf_server_last_error(server)
        elif ctx is not None:
            msg = L.cf_last_error(ctx)
        else:
            msg = b""
        raise CfError(rc, (msg or b"").decode(errors="replace"))


class Params:
    """cf_params plus the edge array it points to (kept alive by this object)."""

    def __init__(self, kind="r", edges=None, autocorr=True, periodic=False, box=0.0, pimax=0.0, npibins=0,
                 refine=(0, 0, 0), ravg=False, weighted=False):
        self.kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        self.edges = np.ascontiguousarray(np.asarray(edges, dtype=np.float64))
        b = (float(box),) * 3 if np.isscalar(box) else tuple(float(v) for v in box)
        self.c = _capi.cf_params(self.kind, int(bool(autocorr)), int(bool(periodic)), (ctypes.c_double * 3)(*b),
                                 self.edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(self.edges) - 1,
                                 float(pimax), int(npibins), (ctypes.c_int * 3)(*refine), int(bool(ravg)),
                                 CF_W_PAIR_PRODUCT if weighted else CF_W_NONE)

    @property
    def nout(self) -> int:
        nb = len(self.edges) - 1
        return nb * (self.c.npibins if self.kind in (CF_DD_RPPI, CF_DD_RPPI_MOCKS) else 1)


def params(**kw) -> Params:
    return Params(**kw)


class Points:
    """cf_points over torch CUDA tensors or numpy arrays (references kept alive)."""

    def __init__(self, x, y, z, w=None):
        self.keep = [x, y, z, w]
        mods = {type(a).__module__.split(".")[0] for a in (x, y, z) if a is not None}
        if "torch" in mods:
            import torch
            arrs = [x, y, z] + ([w] if w is not None else [])
            if not all(isinstance(a, torch.Tensor) for a in arrs):
                raise TypeError("mix of torch and non-torch arrays")
            dt = x.dtype
            if dt not in (torch.float32, torch.float64) or any(a.dtype != dt for a in arrs):
                raise TypeError("coordinates (and weights) must share float32 or float64")
            if not all(a.is_contiguous() for a in arrs):
                raise ValueError("tensors must be contiguous")
            on_dev = int(x.is_cuda)
            if any(a.is_cuda != x.is_cuda for a in arrs):
                raise ValueError("mix of host and device tensors")
            self.dtype = CF_F64 if dt == torch.float64 else CF_F32
            ptr = lambda a: ctypes.c_void_p(a.data_ptr()) if a is not None else None  # noqa: E731
            self.c = _capi.cf_points(ptr(x), ptr(y), ptr(z), ptr(w), x.numel(), self.dtype, on_dev)
        else:
            arrs = [np.ascontiguousarray(np.asarray(a)) for a in (x, y, z)]
            dt = arrs[0].dtype
            if dt not in (np.float32, np.float64):
                raise TypeError("coordinates must be float32 or float64")
            arrs = [a.astype(dt, copy=False) for a in arrs]
            wa = None if w is None else np.ascontiguousarray(np.asarray(w, dtype=dt))
            self.keep = arrs + [wa]
            self.dtype = CF_F64 if dt == np.float64 else CF_F32
            ptr = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None  # noqa: E731
            self.c = _capi.cf_points(ptr(arrs[0]), ptr(arrs[1]), ptr(arrs[2]), ptr(wa), len(arrs[0]), self.dtype, 0)


def points(x, y, z, w=None) -> Points:
    return Points(x, y, z, w)


class _Out:
    """The four result arrays of one catalogue in one host block (the library writes every entry of
    each: npairs, wsum, ravg, wp); the cf_result's pointers are filled from the block's address."""

    def __init__(self, nout: int, nb: int):
        buf = np.empty(3 * nout + nb)
        self.npairs = buf[:nout].view(np.uint64)
        self.wsum = buf[nout:2 * nout]
        self.ravg = buf[2 * nout:3 * nout]
        self.wp = buf[3 * nout:]
        a = buf.ctypes.data
        self.c = _capi.cf_result()
        ctypes.memmove(ctypes.addressof(self.c), (ctypes.c_size_t * 4)(a, a + 8 * nout, a + 16 * nout, a + 24 * nout),
                       ctypes.sizeof(self.c))

    def as_dict(self, p: Params) -> dict:
        d = {"npairs": self.npairs, "wsum": self.wsum}
        if p.c.output_ravg:
            d["ravg"] = self.ravg
        if p.kind == CF_WP:
            d["wp"] = self.wp
        if p.kind in (CF_DD_RPPI, CF_DD_RPPI_MOCKS):
            nb = len(p.edges) - 1
            for k in ("npairs", "wsum", "ravg"):
                if k in d:
                    d[k] = d[k].reshape(nb, p.c.npibins)
        return d


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def cf_create(device: int = 0, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(_capi.lib().cf_create(ctypes.byref(h), int(device), _stream_handle(stream)))
    return h.value


def cf_destroy(ctx: int) -> None:
    _check(_capi.lib().cf_destroy(ctx))


def cf_last_error(ctx: int) -> str:
    return (_capi.lib().cf_last_error(ctx) or b"").decode()


def cf_set_option(ctx: int, option: int, value: int) -> None:
    _check(_capi.lib().cf_set_option(ctx, int(option), int(value)), ctx)


def cf_count(ctx: int, p: Params, d1: Points, d2: Optional[Points] = None) -> dict:
    out = _Out(p.nout, len(p.edges) - 1)
    _check(_capi.lib().cf_count(ctx, ctypes.byref(p.c), ctypes.byref(d1.c), ctypes.byref(d2.c) if d2 else None,
                                ctypes.byref(out.c)), ctx)
    return out.as_dict(p)


def cf_batch_count(ctx: int, p: Params, cats: Sequence[Points]) -> list:
    n = len(cats)
    arr = (_capi.cf_points * n)(*[c.c for c in cats])
    outs = [_Out(p.nout, len(p.edges) - 1) for _ in range(n)]
    res = (_capi.cf_result * n)(*[o.c for o in outs])
    _check(_capi.lib().cf_batch_count(ctx, ctypes.byref(p.c), arr, n, res), ctx)
    return [o.as_dict(p) for o in outs]


def cf_get_stats(ctx: int) -> dict:
    s = _capi.cf_stats()
    _check(_capi.lib().cf_get_stats(ctx, ctypes.byref(s)), ctx)
    return {f: (list(getattr(s, f)) if f in ("grid", "refine") else getattr(s, f)) for f, _ in s._fields_}


# ---- serving (continuous batching) ----
_server_keep = {}


def cf_server_start(device: int, p: Params, mem_budget_bytes: int, max_slots: int) -> int:
    h = ctypes.c_void_p()
    _check(_capi.lib().cf_server_start(ctypes.byref(h), int(device), ctypes.byref(p.c), int(mem_budget_bytes),
                                       int(max_slots)))
    _server_keep[h.value] = {"params": p}
    return h.value


def cf_server_submit(server: int, p: Params, cat: Points) -> int:
    """Queue one catalogue; returns its ticket.  The catalogue arrays must stay alive until the
    ticket is polled (the binding keeps a reference)."""
    out = _Out(p.nout, len(p.edges) - 1)
    t = ctypes.c_uint64()
    _check(_capi.lib().cf_server_submit(server, ctypes.byref(cat.c), ctypes.byref(out.c), ctypes.byref(t)),
           server=server)
    _server_keep[server][t.value] = (out, cat)
    return t.value


def cf_server_poll(server: int, ticket: int, timeout_ms: int = 0):
    """Returns the result dict when done, None while busy (timeout_ms == 0) or on timeout."""
    rc = _capi.lib().cf_server_poll(server, ctypes.c_uint64(ticket), int(timeout_ms))
    if rc in (_capi.CF_ERR_BUSY, _capi.CF_ERR_TIMEOUT):
        return None
    keep = _server_keep[server].pop(ticket, None)
    _check(rc, server=server)
    return keep[0].as_dict(_server_keep[server]["params"])


def cf_server_cancel(server: int, ticket: int) -> bool:
    """Withdraw a request.  True when the library no longer uses its buffers: it was queued and is
    withdrawn (cf_server_poll then raises CF_ERR_CANCELLED), or it had already finished (poll
    returns its result).  False when it is in a wave on the GPU: it runs to the end and
    cf_server_poll returns its result."""
    rc = _capi.lib().cf_server_cancel(server, ctypes.c_uint64(ticket))
    if rc == _capi.CF_ERR_BUSY:
        return False
    _check(rc, server=server)
    return True


def cf_server_stop(server: int) -> None:
    _check(_capi.lib().cf_server_stop(server))
    _server_keep.pop(server, None)


def cf_server_last_error(server: int) -> str:
    return (_capi.lib().cf_server_last_error(server) or b"").decode()


def cf_batch_capture(ctx: int, p: Params, cats: Sequence[Points]) -> None:
    n = len(cats)
    arr = (_capi.cf_points * n)(*[c.c for c in cats])
    _check(_capi.lib().cf_batch_capture(ctx, ctypes.byref(p.c), arr, n), ctx)


def cf_batch_replay(ctx: int, p: Params, n: int) -> list:
    outs = [_Out(p.nout, len(p.edges) - 1) for _ in range(n)]
    res = (_capi.cf_result * n)(*[o.c for o in outs])
    _check(_capi.lib().cf_batch_replay(ctx, res, n), ctx)
    return [o.as_dict(p) for o in outs]


def cf_plan_probe(p: Params, bbox, npoints: int, any_f64: bool = False, which: int = 0, values=None) -> dict:
    """Host-only: the plan cf_count would build (grid, bands, table sizes) and, optionally, the
    table classification of FP32 `values` (see include/cf.h)."""
    info = _capi.cf_plan_info()
    nb = len(p.edges) - 1
    npi = max(1, p.c.npibins)
    br = np.zeros(nb + 1)
    bp = np.zeros(npi + 1)
    bb = np.ascontiguousarray(np.asarray(bbox, dtype=np.float64))
    D = ctypes.POINTER(ctypes.c_double)
    if values is None:
        vals = np.zeros(0, dtype=np.float32)
    else:
        vals = np.ascontiguousarray(np.asarray(values, dtype=np.float32))
    cls = np.zeros(len(vals), dtype=np.uint32)
    rc = _capi.lib().cf_plan_probe(ctypes.byref(p.c), bb.ctypes.data_as(D), int(npoints), int(bool(any_f64)),
                                   ctypes.byref(info), br.ctypes.data_as(D), bp.ctypes.data_as(D), int(which),
                                   vals.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(vals),
                                   cls.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    _check(rc)
    out = {f: (list(getattr(info, f)) if hasattr(getattr(info, f), "__len__") else getattr(info, f))
           for f, _ in info._fields_}
    out["bands_r"] = br
    out["bands_p"] = bp[: p.c.npibins + 1] if p.kind in (CF_DD_RPPI, CF_WP, CF_DD_RPPI_MOCKS) else np.zeros(0)
    out["classes"] = cls
    return out


def cf_count_noalloc(p: Params, d1: Points, d2: Optional[Points], npairs, wsum=None, ravg=None, stream=None) -> None:
    """Allocation-free count into caller-owned device tensors (see include/cf.h): for callers that
    cannot allocate device memory.  npairs is int64 (the counts' bits), wsum and ravg float64, each
    a contiguous tensor on the current CUDA device with at least p.nout elements (ValueError
    otherwise: the library writes p.nout entries through the raw pointers).  Enqueued on `stream`;
    returns without waiting."""
    import torch
    dev = torch.cuda.current_device()

    def ptr(t, name, dtype):
        if t is None:
            return None
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device.index != dev:
            raise ValueError(f"{name} must be a tensor on the current CUDA device (cuda:{dev})")
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}, not {t.dtype}")
        if not t.is_contiguous() or t.numel() < p.nout:
            raise ValueError(f"{name} must be contiguous with at least {p.nout} elements")
        return ctypes.c_void_p(t.data_ptr())

    out = (ptr(npairs, "npairs", torch.int64), ptr(wsum, "wsum", torch.float64), ptr(ravg, "ravg", torch.float64))
    rc = _capi.lib().cf_count_noalloc(ctypes.byref(p.c), ctypes.byref(d1.c), ctypes.byref(d2.c) if d2 else None,
                                      *out, _stream_handle(stream))
    _check(rc)
