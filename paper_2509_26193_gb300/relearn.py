"""Thin ctypes binding of librelearn (include/relearn.h), same names as the C ABI.

Only argument marshalling lives here: tensors are checked (device, dtype,
contiguity, length) and their device pointers passed through; every step of
the connectivity update runs in the library's CUDA kernels. There is no CPU
fallback: if ``_lib/librelearn.so`` is missing, the first call raises.
PyTorch provides device memory and the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librelearn.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "relearn.h")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_CAPACITY, ERR_TIMEOUT, ERR_STATE = range(7)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "CAPACITY", 5: "TIMEOUT",
                6: "STATE"}
FLAG_DIAG = 1
FLAG_TIMING = 2
FLAG_REGROUP = 4
FLAG_COUNT = 8

_lock = threading.Lock()
_lib = None


class RelearnError(RuntimeError):
    def __init__(self, status, where, msg=""):
        self.status = status
        super().__init__(f"{where}: RELEARN_ERR_{STATUS_NAMES.get(status, status)} {msg}".strip())


class relearn_params(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_float), ("theta", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("step", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("search_group", ctypes.c_uint32), ("net_sigma", ctypes.c_void_p),
                ("net_theta", ctypes.c_void_p)]


class relearn_update_stats(ctypes.Structure):
    _fields_ = [("searches", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("requests_declined", ctypes.c_int64), ("formed", ctypes.c_int64),
                ("synapses", ctypes.c_int64), ("ms_reduce", ctypes.c_float),
                ("ms_search", ctypes.c_float), ("ms_search_kernel", ctypes.c_float),
                ("ms_accept", ctypes.c_float), ("ms_apply", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("reserved", ctypes.c_int32),
                ("searches_total", ctypes.c_int64), ("evals_total", ctypes.c_int64),
                ("walk_steps_total", ctypes.c_int64), ("length_evals_total", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "relearn_create": [ctypes.POINTER(_P), ctypes.c_int, _I64, _I64, _I64],
    "relearn_create_batched": [ctypes.POINTER(_P), ctypes.c_int, _I64, _I64, _I64,
                               ctypes.c_int32],
    "relearn_destroy": [_P],
    "relearn_build_octree": [_P, _I64, _P, _P, _P, _P, _P, _P, _P],
    "relearn_build_octree_batch": [_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P],
    "relearn_update_connectivity": [_P, ctypes.POINTER(relearn_params), _P, _P, _P,
                                    ctypes.POINTER(relearn_update_stats), _P],
    "relearn_delete_synapses": [_P, ctypes.POINTER(relearn_params), _P, _P, _P, _P,
                                ctypes.POINTER(_I64), _P],
    "relearn_deliver_spikes": [_P, _P, _P, _P],
    "relearn_mean_length": [_P, ctypes.POINTER(relearn_params), _P, _P, _P, _P, _P],
    "relearn_debug_stall_scan": [_P, ctypes.c_int64],
    "relearn_update_connectivity_typed": [_P, ctypes.POINTER(relearn_params), _P, _P, _P, _P,
                                          ctypes.POINTER(relearn_update_stats), _P],
    "relearn_mean_length_backward": [_P, _P, _P, _P, _P, _P, _P, _P, _P],
    "relearn_deliver_rates": [_P, _P, ctypes.c_uint64, ctypes.c_uint64, _P, _P],
    "relearn_get_synapses": [_P, _I64, ctypes.POINTER(_I64), _P, _P, _P],
    "relearn_set_synapses": [_P, _I64, _P, _P, _P],
    "relearn_get_requests": [_P, _I64, ctypes.POINTER(_I64), _P, _P],
    "relearn_get_search_diag": [_P, _I64, ctypes.POINTER(_I64), _P, _P, _P],
    "relearn_get_tree": [_P, _I64, ctypes.POINTER(_I64)] + [_P] * 10,
    "relearn_philox4x32_10": [_P, _P, _P, _I64, _P],
    "relearn_get_last_stats": [_P, ctypes.POINTER(relearn_update_stats)],
    "relearn_collect_search_times": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)],
    "relearn_launch_count": [ctypes.POINTER(_I64)],
    "relearn_morton_order_noalloc": [_I64, _P, _P, _P, _P, _P, _P, _P, _P],
    "relearn_peak_probe": [ctypes.c_int32, _I64, _P, _I64, ctypes.POINTER(_I64), _P],
    "relearn_last_error": [_P, ctypes.POINTER(ctypes.c_char_p)],
}


def header_functions(path=HEADER):
    """Names of the functions declared in include/relearn.h."""
    text = open(path).read()
    return sorted(set(re.findall(r"^relearn_status\s+(relearn_\w+)\s*\(", text, re.M)))


def lib():
    """Load librelearn.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with paper_2509_26193_gb300.build.build() "
                    "(there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            _lib = L
    return _lib


# --------------------------------------------------------------------- helpers
def _torch():
    import torch
    return torch


def _dev_ptr(t, dtype, n, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name}: needs {n} elements, has {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Context:
    """Handle of one relearn_ctx (owns its device scratch)."""

    def __init__(self, handle, device, max_neurons, max_synapses, max_searches):
        self.handle = handle
        self.device = device
        self.max_neurons = max_neurons
        self.max_synapses = max_synapses
        self.max_searches = max_searches
        self.n = 0
        self.num_networks = 1
        self.keep = ()  # device arrays a params struct points at (per-network sigma/theta)

    def close(self):
        if self.handle:
            lib().relearn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _raise(ctx, status, where):
    if status == OK:
        return
    msg = ""
    if ctx is not None and ctx.handle:
        m = ctypes.c_char_p()
        lib().relearn_last_error(ctx.handle, ctypes.byref(m))
        msg = (m.value or b"").decode(errors="replace")
    raise RelearnError(status, where, msg)


def params(sigma, theta, seed, step, flags=0, search_group=0, net_sigma=None, net_theta=None):
    """net_sigma / net_theta: optional float32 CUDA tensors, one value per network; the
    caller keeps them alive while the params are in use."""
    torch = _torch() if (net_sigma is not None or net_theta is not None) else None
    ps = None if net_sigma is None else _dev_ptr(net_sigma, torch.float32, None, "net_sigma")
    pt = None if net_theta is None else _dev_ptr(net_theta, torch.float32, None, "net_theta")
    return relearn_params(float(sigma), float(theta), int(seed), int(step), int(flags),
                          int(search_group), ps, pt)


# ------------------------------------------------------------------ entry points
def relearn_create(max_neurons, max_synapses, max_searches=0, device=None):
    torch = _torch()
    dev = torch.cuda.current_device() if device is None else int(device)
    h = ctypes.c_void_p()
    st = lib().relearn_create(ctypes.byref(h), dev, int(max_neurons), int(max_synapses),
                              int(max_searches))
    if st != OK:
        raise RelearnError(st, "relearn_create")
    return Context(h, dev, int(max_neurons), int(max_synapses), int(max_searches))


def relearn_create_batched(max_neurons, max_synapses, max_networks, max_searches=0, device=None):
    torch = _torch()
    dev = torch.cuda.current_device() if device is None else int(device)
    h = ctypes.c_void_p()
    st = lib().relearn_create_batched(ctypes.byref(h), dev, int(max_neurons), int(max_synapses),
                                      int(max_searches), int(max_networks))
    if st != OK:
        raise RelearnError(st, "relearn_create_batched")
    return Context(h, dev, int(max_neurons), int(max_synapses), int(max_searches))


def relearn_destroy(ctx):
    ctx.close()


def _box_corners(box_lo, box_hi):
    """Host float32[3] copies of a caller-given domain box (both corners or none)."""
    if (box_lo is None) != (box_hi is None):
        raise ValueError("give both box corners or none")
    if box_lo is None:
        return None, None
    lo = np.ascontiguousarray(box_lo, np.float32).ravel()
    hi = np.ascontiguousarray(box_hi, np.float32).ravel()
    if lo.size != 3 or hi.size != 3:
        raise ValueError("each box corner holds 3 floats (x, y, z)")
    return lo, hi


def relearn_build_octree(ctx, x, y, z, vac_de=None, box_lo=None, box_hi=None, stream=None):
    torch = _torch()
    n = x.numel()
    px = _dev_ptr(x, torch.float32, n, "x")
    py = _dev_ptr(y, torch.float32, n, "y")
    pz = _dev_ptr(z, torch.float32, n, "z")
    pv = None if vac_de is None else _dev_ptr(vac_de, torch.int32, n, "vac_de")
    lo, hi = _box_corners(box_lo, box_hi)
    st = lib().relearn_build_octree(ctx.handle, n, px, py, pz, pv, _np_ptr(lo), _np_ptr(hi),
                                    _stream(stream))
    _raise(ctx, st, "relearn_build_octree")
    ctx.n = n
    ctx.num_networks = 1


def relearn_update_connectivity_typed(ctx, prm, vac_ax, vac_de_exc, vac_de_inh, type_,
                                      stats=False, stream=None):
    torch = _torch()
    n = ctx.n
    a = _dev_ptr(vac_ax, torch.int32, n, "vac_ax")
    de = _dev_ptr(vac_de_exc, torch.int32, n, "vac_de_exc")
    di = _dev_ptr(vac_de_inh, torch.int32, n, "vac_de_inh")
    t = _dev_ptr(type_, torch.uint8, n, "type")
    s = relearn_update_stats() if stats else None
    st = lib().relearn_update_connectivity_typed(ctx.handle, ctypes.byref(prm), a, de, di, t,
                                                 ctypes.byref(s) if s is not None else None,
                                                 _stream(stream))
    _raise(ctx, st, "relearn_update_connectivity_typed")
    return s.as_dict() if s is not None else None


def relearn_debug_stall_scan(ctx, tile):
    """Testing hook: in the next bottom-up update of ctx, prefix tile `tile` publishes
    nothing, so that update's bounded waits run out (RELEARN_ERR_TIMEOUT)."""
    _raise(ctx, lib().relearn_debug_stall_scan(ctx.handle, int(tile)),
           "relearn_debug_stall_scan")


def relearn_build_octree_batch(ctx, offsets, x, y, z, vac_de=None, stream=None):
    """offsets: host int64 sequence of num_networks + 1 entries (0 .. n)."""
    torch = _torch()
    off = np.ascontiguousarray(offsets, np.int64)
    if off.ndim != 1 or off.size < 2:
        raise ValueError("offsets: need num_networks + 1 entries")
    n = int(off[-1])
    if x.numel() < n:
        raise ValueError("x: fewer positions than offsets[-1]")
    px = _dev_ptr(x, torch.float32, n, "x")
    py = _dev_ptr(y, torch.float32, n, "y")
    pz = _dev_ptr(z, torch.float32, n, "z")
    pv = None if vac_de is None else _dev_ptr(vac_de, torch.int32, n, "vac_de")
    st = lib().relearn_build_octree_batch(ctx.handle, int(off.size - 1), _np_ptr(off), px, py,
                                          pz, pv, _stream(stream))
    _raise(ctx, st, "relearn_build_octree_batch")
    ctx.n = n
    ctx.num_networks = int(off.size - 1)


def relearn_update_connectivity(ctx, prm, vac_ax, vac_de, type_, stats=False, stream=None):
    torch = _torch()
    n = ctx.n
    a = _dev_ptr(vac_ax, torch.int32, n, "vac_ax")
    d = _dev_ptr(vac_de, torch.int32, n, "vac_de")
    t = _dev_ptr(type_, torch.uint8, n, "type")
    s = relearn_update_stats() if stats else None
    st = lib().relearn_update_connectivity(ctx.handle, ctypes.byref(prm), a, d, t,
                                           ctypes.byref(s) if s is not None else None,
                                           _stream(stream))
    _raise(ctx, st, "relearn_update_connectivity")
    return s.as_dict() if s is not None else None


def relearn_delete_synapses(ctx, prm, retract_ax, retract_de, vac_ax, vac_de, count=False,
                            stream=None):
    torch = _torch()
    n = ctx.n
    ra = _dev_ptr(retract_ax, torch.int32, n, "retract_ax")
    rd = _dev_ptr(retract_de, torch.int32, n, "retract_de")
    a = _dev_ptr(vac_ax, torch.int32, n, "vac_ax")
    d = _dev_ptr(vac_de, torch.int32, n, "vac_de")
    b = ctypes.c_int64(0)
    st = lib().relearn_delete_synapses(ctx.handle, ctypes.byref(prm), ra, rd, a, d,
                                       ctypes.byref(b) if count else None, _stream(stream))
    _raise(ctx, st, "relearn_delete_synapses")
    return b.value if count else None


def relearn_mean_length(ctx, prm, vac_ax, vac_de, mean, ell=None, stream=None):
    """mean: float64 CUDA tensor (1 element), written; ell: float32 [n] or None."""
    torch = _torch()
    n = ctx.n
    a = _dev_ptr(vac_ax, torch.int32, n, "vac_ax")
    d = _dev_ptr(vac_de, torch.int32, n, "vac_de")
    m = _dev_ptr(mean, torch.float64, 1, "mean")
    e = None if ell is None else _dev_ptr(ell, torch.float32, n, "ell")
    st = lib().relearn_mean_length(ctx.handle, ctypes.byref(prm), a, d, e, m, _stream(stream))
    _raise(ctx, st, "relearn_mean_length")


def relearn_mean_length_backward(ctx, vac_ax, vac_de, gx, gy, gz, grad_mean=None, gsigma=None,
                                 stream=None):
    torch = _torch()
    n = ctx.n
    a = _dev_ptr(vac_ax, torch.int32, n, "vac_ax")
    d = _dev_ptr(vac_de, torch.int32, n, "vac_de")
    g = [_dev_ptr(t, torch.float32, n, name) for t, name in ((gx, "gx"), (gy, "gy"), (gz, "gz"))]
    gm = None if grad_mean is None else _dev_ptr(grad_mean, torch.float64, 1, "grad_mean")
    gs = None if gsigma is None else _dev_ptr(gsigma, torch.float64, 1, "gsigma")
    st = lib().relearn_mean_length_backward(ctx.handle, a, d, gm, *g, gs, _stream(stream))
    _raise(ctx, st, "relearn_mean_length_backward")


def relearn_deliver_spikes(ctx, spiked, out, stream=None):
    torch = _torch()
    n = ctx.n
    s = _dev_ptr(spiked, torch.uint8, n, "spiked")
    o = _dev_ptr(out, torch.int32, n, "input")
    st = lib().relearn_deliver_spikes(ctx.handle, s, o, _stream(stream))
    _raise(ctx, st, "relearn_deliver_spikes")


def relearn_deliver_rates(ctx, rate, seed, step, out, stream=None):
    torch = _torch()
    n = ctx.n
    r = _dev_ptr(rate, torch.float32, n, "rate")
    o = _dev_ptr(out, torch.int32, n, "input")
    st = lib().relearn_deliver_rates(ctx.handle, r, int(seed), int(step), o, _stream(stream))
    _raise(ctx, st, "relearn_deliver_rates")


def relearn_get_synapses(ctx):
    cnt = ctypes.c_int64(0)
    st = lib().relearn_get_synapses(ctx.handle, 0, ctypes.byref(cnt), None, None, None)
    _raise(ctx, st, "relearn_get_synapses")
    m = cnt.value
    src = np.zeros(m, np.int32)
    tgt = np.zeros(m, np.int32)
    sign = np.zeros(m, np.int8)
    st = lib().relearn_get_synapses(ctx.handle, m, ctypes.byref(cnt), _np_ptr(src), _np_ptr(tgt),
                                    _np_ptr(sign))
    _raise(ctx, st, "relearn_get_synapses")
    return src, tgt, sign


def relearn_set_synapses(ctx, src, tgt, sign):
    src = np.ascontiguousarray(src, np.int32)
    tgt = np.ascontiguousarray(tgt, np.int32)
    sign = np.ascontiguousarray(sign, np.int8)
    st = lib().relearn_set_synapses(ctx.handle, src.shape[0], _np_ptr(src), _np_ptr(tgt),
                                    _np_ptr(sign))
    _raise(ctx, st, "relearn_set_synapses")


def relearn_get_requests(ctx):
    cnt = ctypes.c_int64(0)
    st = lib().relearn_get_requests(ctx.handle, 0, ctypes.byref(cnt), None, None)
    _raise(ctx, st, "relearn_get_requests")
    q = cnt.value
    tgt = np.zeros(q, np.int32)
    acc = np.zeros(q, np.uint8)
    st = lib().relearn_get_requests(ctx.handle, q, ctypes.byref(cnt), _np_ptr(tgt), _np_ptr(acc))
    _raise(ctx, st, "relearn_get_requests")
    return tgt, acc


def relearn_get_search_diag(ctx):
    cnt = ctypes.c_int64(0)
    st = lib().relearn_get_search_diag(ctx.handle, 0, ctypes.byref(cnt), None, None, None)
    _raise(ctx, st, "relearn_get_search_diag")
    q = cnt.value
    lns = np.zeros(q, np.float64)
    ev = np.zeros(q, np.int32)
    rs = np.zeros(q, np.int32)
    st = lib().relearn_get_search_diag(ctx.handle, q, ctypes.byref(cnt), _np_ptr(lns),
                                       _np_ptr(ev), _np_ptr(rs))
    _raise(ctx, st, "relearn_get_search_diag")
    return {"ln_s0": lns, "evals": ev, "restarts": rs}


def relearn_get_tree(ctx):
    cnt = ctypes.c_int64(0)
    st = lib().relearn_get_tree(ctx.handle, 0, ctypes.byref(cnt), *([None] * 10))
    _raise(ctx, st, "relearn_get_tree")
    m = cnt.value
    out = {k: np.zeros(m, np.int32) for k in ("depth", "first", "size", "is_leaf", "neuron",
                                               "count")}
    out.update({k: np.zeros(m, np.float32) for k in ("cx", "cy", "cz")})
    perm = np.zeros(ctx.n, np.int32)
    st = lib().relearn_get_tree(ctx.handle, m, ctypes.byref(cnt),
                                *(_np_ptr(out[k]) for k in ("depth", "first", "size", "is_leaf",
                                                            "neuron", "count", "cx", "cy", "cz")),
                                _np_ptr(perm))
    _raise(ctx, st, "relearn_get_tree")
    out["perm"] = perm
    return out


def relearn_philox4x32_10(ctr, key, out, stream=None):
    torch = _torch()
    n = ctr.numel() // 4
    c = _dev_ptr(ctr, torch.int32, 4 * n, "ctr")
    k = _dev_ptr(key, torch.int32, 2 * n, "key")
    o = _dev_ptr(out, torch.int32, 4 * n, "out")
    st = lib().relearn_philox4x32_10(c, k, o, n, _stream(stream))
    _raise(None, st, "relearn_philox4x32_10")


def relearn_get_last_stats(ctx):
    s = relearn_update_stats()
    st = lib().relearn_get_last_stats(ctx.handle, ctypes.byref(s))
    _raise(ctx, st, "relearn_get_last_stats")
    return s.as_dict()


def relearn_collect_search_times(ctx):
    ms = ctypes.c_double(0.0)
    k = ctypes.c_int64(0)
    st = lib().relearn_collect_search_times(ctx.handle, ctypes.byref(ms), ctypes.byref(k))
    _raise(ctx, st, "relearn_collect_search_times")
    return ms.value, k.value


def relearn_launch_count():
    c = ctypes.c_int64(0)
    st = lib().relearn_launch_count(ctypes.byref(c))
    _raise(None, st, "relearn_launch_count")
    return c.value


def relearn_morton_order_noalloc(x, y, z, codes, perm, box_lo=None, box_hi=None, stream=None):
    """Morton codes and order without any device allocation inside the library; the
    caller provides `codes` (uint32 viewed as int32) and `perm` (int32) on the device."""
    torch = _torch()
    n = x.numel()
    px = _dev_ptr(x, torch.float32, n, "x")
    py = _dev_ptr(y, torch.float32, n, "y")
    pz = _dev_ptr(z, torch.float32, n, "z")
    pc = _dev_ptr(codes, torch.int32, n, "codes")
    pp = _dev_ptr(perm, torch.int32, n, "perm")
    lo, hi = _box_corners(box_lo, box_hi)
    st = lib().relearn_morton_order_noalloc(n, px, py, pz, _np_ptr(lo), _np_ptr(hi), pc, pp,
                                            _stream(stream))
    _raise(None, st, "relearn_morton_order_noalloc")


PROBE_FMA, PROBE_EX2, PROBE_L2, PROBE_FMA2 = 1, 2, 3, 4


def relearn_peak_probe(kind, iters, buf, stream=None):
    """Launches one measurement probe on the current stream (see relearn.h); returns the
    work of the launch (FMAs, ex2 evaluations or bytes read). The caller times it."""
    torch = _torch()
    pb = _dev_ptr(buf, torch.float32, buf.numel(), "buf")
    ops = ctypes.c_int64()
    st = lib().relearn_peak_probe(int(kind), int(iters), pb, buf.numel(), ctypes.byref(ops),
                                  _stream(stream))
    _raise(None, st, "relearn_peak_probe")
    return int(ops.value)


def relearn_last_error(ctx):
    m = ctypes.c_char_p()
    st = lib().relearn_last_error(ctx.handle, ctypes.byref(m))
    return st, (m.value or b"").decode(errors="replace")
