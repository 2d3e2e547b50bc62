"""FP64 CPU oracle of the MSP connectivity update (arXiv 2509.26193, Sec. III).

TEST INFRASTRUCTURE ONLY. The oracle checks the CUDA path and shares no code
with it. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import this package; the product path never
does.

The arithmetic lives in ``oracle.c`` (plain C, FP64); this module compiles it
with gcc and wraps it with ctypes + numpy. Functions and the paper passages they
follow are listed in the header of ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_lib/liboracle.so`` (OpenMP when available)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-Wall", "-Wno-unused-function"]
    tmp = _LIB + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class SearchDiag(ctypes.Structure):
    _fields_ = [("target", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("evals", ctypes.c_int64), ("expansions", ctypes.c_int64),
                ("evals_zero", ctypes.c_int64), ("frontier0", ctypes.c_int64),
                ("ln_s0", ctypes.c_double), ("margin_ac", ctypes.c_double),
                ("margin_draw", ctypes.c_double)]


DIAG_DTYPE = np.dtype([("target", np.int32), ("restarts", np.int32), ("evals", np.int64),
                       ("expansions", np.int64), ("evals_zero", np.int64),
                       ("frontier0", np.int64), ("ln_s0", np.float64),
                       ("margin_ac", np.float64), ("margin_draw", np.float64)])
assert DIAG_DTYPE.itemsize == ctypes.sizeof(SearchDiag)

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_I32 = ctypes.c_int32
_D = ctypes.c_double


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            sig = {
                "orc_philox4x32_10": (None, [_P, _P, _P]),
                "orc_morton": (None, [_I64, _P, _P, _P, _P, _P, _P, _P, _P]),
                "orc_tree_build": (_P, [_I64, _P, _P, _P, _P, _P]),
                "orc_tree_free": (None, [_P]),
                "orc_tree_set_id_base": (None, [_P, _I64]),
                "orc_tree_num_nodes": (_I64, [_P]),
                "orc_tree_box": (None, [_P, _P, _P]),
                "orc_tree_canonical_order": (None, [_P, _P]),
                "orc_tree_reduce": (None, [_P, _P]),
                "orc_tree_export": (_I64, [_P, ctypes.c_int] + [_P] * 9),
                "orc_search": (_I32, [_P, _D, _D, _U64, _U64, _I32, _I32, _P]),
                "orc_search_batch": (None, [_P, _D, _D, _U64, _U64, _I64, _P, _P, _P, _P,
                                            ctypes.c_int]),
                "orc_openmp_available": (ctypes.c_int, []),
                "orc_search_marginals": (None, [_P, _D, _D, _I32, _P]),
                "orc_request_priority": (ctypes.c_uint32, [_U64, _U64, _I32, _I32]),
                "orc_accept": (None, [_I64, _I64, _P, _P, _P, _P, _U64, _U64, _P]),
                "orc_apply": (_I64, [_I64, _P, _P, _P, _P, _P, _P, _P, _I64, _P, _P, _P]),
                "orc_delete": (_I64, [_I64, _P, _P, _P, _P, _U64, _U64, _P, _P, _P, _P]),
                "orc_deliver_spikes": (None, [_I64, _I64, _P, _P, _P, _P, _P]),
                "orc_deliver_rates": (None, [_I64, _I64, _P, _P, _P, _P, _U64, _U64, _P]),
                "orc_mean_length": (_D, [_P, _D, _D, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                         _P, ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------- RNG
def philox4x32_10(ctr, key):
    """Philox4x32-10 block: 4 uint32 counter words, 2 uint32 key words -> 4 words."""
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


# ------------------------------------------------------------------------ Morton
def morton(x, y, z, box_lo=None, box_hi=None):
    """30-bit Morton codes of FP32 positions; returns (codes, lo, hi)."""
    x, y, z = (_c(a, np.float32) for a in (x, y, z))
    n = x.shape[0]
    codes = np.zeros(n, np.uint32)
    lo = np.zeros(3, np.float32)
    hi = np.zeros(3, np.float32)
    bl = None if box_lo is None else _c(box_lo, np.float32)
    bh = None if box_hi is None else _c(box_hi, np.float32)
    lib().orc_morton(n, _p(x), _p(y), _p(z), _p(bl), _p(bh), _p(codes), _p(lo), _p(hi))
    return codes, lo, hi


# -------------------------------------------------------------------------- tree
class Tree:
    """Pointer octree over the positions (Sec. III-B "Spatial octree")."""

    def __init__(self, x, y, z, box_lo=None, box_hi=None, id_base=0):
        """id_base: global id of neuron 0 when the tree holds one network of a batch
        (the search draws are keyed by global ids); results stay local ids."""
        self._x, self._y, self._z = (_c(a, np.float32) for a in (x, y, z))
        self.n = self._x.shape[0]
        bl = None if box_lo is None else _c(box_lo, np.float32)
        bh = None if box_hi is None else _c(box_hi, np.float32)
        self._h = lib().orc_tree_build(self.n, _p(self._x), _p(self._y), _p(self._z),
                                       _p(bl), _p(bh))
        self.id_base = int(id_base)
        if self.id_base:
            lib().orc_tree_set_id_base(self._h, self.id_base)

    def close(self):
        if self._h:
            lib().orc_tree_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_nodes(self):
        return int(lib().orc_tree_num_nodes(self._h))

    def box(self):
        lo = np.zeros(3, np.float32)
        hi = np.zeros(3, np.float32)
        lib().orc_tree_box(self._h, _p(lo), _p(hi))
        return lo, hi

    def canonical_order(self):
        perm = np.zeros(self.n, np.int32)
        lib().orc_tree_canonical_order(self._h, _p(perm))
        return perm

    def reduce(self, vac_de):
        """Bottom-up count / centroid update (Sec. III-B "Division of work")."""
        self._vac_de = _c(vac_de, np.int32)
        lib().orc_tree_reduce(self._h, _p(self._vac_de))

    def export(self, compressed=False):
        """Nodes in pre-order as a dict of arrays."""
        m = self.num_nodes
        out = {k: np.zeros(m, np.int32) for k in ("depth", "first", "size", "is_leaf", "neuron")}
        out.update({k: np.zeros(m, np.float64) for k in ("count", "cx", "cy", "cz")})
        k = lib().orc_tree_export(self._h, 1 if compressed else 0,
                                  *(_p(out[name]) for name in ("depth", "first", "size",
                                                               "is_leaf", "neuron", "count",
                                                               "cx", "cy", "cz")))
        return {name: arr[:k].copy() for name, arr in out.items()}

    # ---------------------------------------------------------------- search
    def search(self, sigma, theta, seed, step, i, e):
        d = SearchDiag()
        lib().orc_search(self._h, sigma, theta, seed, step, int(i), int(e), ctypes.byref(d))
        return {name: getattr(d, name) for name, _ in SearchDiag._fields_}

    def search_batch(self, sigma, theta, seed, step, qi, qe, threads=1):
        qi = _c(qi, np.int32)
        qe = _c(qe, np.int32)
        nq = qi.shape[0]
        tgt = np.zeros(nq, np.int32)
        diag = np.zeros(nq, DIAG_DTYPE)
        lib().orc_search_batch(self._h, sigma, theta, seed, step, nq, _p(qi), _p(qe),
                               _p(tgt), _p(diag), int(threads))
        return tgt, diag

    def marginals(self, sigma, theta, i):
        """Exact outcome distribution of one search; entry n = failure."""
        probs = np.zeros(self.n + 1, np.float64)
        lib().orc_search_marginals(self._h, sigma, theta, int(i), _p(probs))
        return probs


def openmp_available():
    return bool(lib().orc_openmp_available())


# ---------------------------------------------------------------- queries
def queries(vac_ax):
    """(neuron, element) pairs in canonical order: neuron id, then element."""
    vac_ax = np.maximum(np.asarray(vac_ax, np.int64), 0)
    qi = np.repeat(np.arange(vac_ax.shape[0], dtype=np.int32), vac_ax)
    starts = np.cumsum(vac_ax) - vac_ax
    qe = (np.arange(qi.shape[0], dtype=np.int64) - np.repeat(starts, vac_ax)).astype(np.int32)
    return qi, qe


# ---------------------------------------------------------- accept / apply
def request_priority(seed, step, src, elem):
    return int(lib().orc_request_priority(seed, step, int(src), int(elem)))


def accept(n, src, elem, tgt, vac_de, seed, step):
    src, elem, tgt = (_c(a, np.int32) for a in (src, elem, tgt))
    vac_de = _c(vac_de, np.int32)
    acc = np.zeros(src.shape[0], np.uint8)
    lib().orc_accept(n, src.shape[0], _p(src), _p(elem), _p(tgt), _p(vac_de), seed, step,
                     _p(acc))
    return acc


class Synapses:
    """Canonical synapse multiset (sorted by source, then target)."""

    def __init__(self, capacity, src=None, tgt=None, sign=None):
        self.cap = int(capacity)
        self.src = np.zeros(max(self.cap, 1), np.int32)
        self.tgt = np.zeros(max(self.cap, 1), np.int32)
        self.sign = np.zeros(max(self.cap, 1), np.int8)
        self.count = 0
        if src is not None:
            m = len(src)
            order = np.lexsort((np.asarray(sign), np.asarray(tgt), np.asarray(src)))
            self.src[:m] = np.asarray(src)[order]
            self.tgt[:m] = np.asarray(tgt)[order]
            self.sign[:m] = np.asarray(sign)[order]
            self.count = m

    def arrays(self):
        m = self.count
        return self.src[:m].copy(), self.tgt[:m].copy(), self.sign[:m].copy()


def apply(src, tgt, accepted, type_, vac_ax, vac_de, syn: Synapses):
    """Apply accepted requests in place (vac_ax, vac_de, syn); returns synapses formed."""
    src, tgt = _c(src, np.int32), _c(tgt, np.int32)
    accepted = _c(accepted, np.uint8)
    type_ = _c(type_, np.uint8)
    cnt = ctypes.c_int64(syn.count)
    formed = lib().orc_apply(src.shape[0], _p(src), _p(tgt), _p(accepted), _p(type_),
                             _p(vac_ax), _p(vac_de), ctypes.byref(cnt), syn.cap,
                             _p(syn.src), _p(syn.tgt), _p(syn.sign))
    if formed < 0:
        raise RuntimeError("synapse capacity exceeded")
    syn.count = cnt.value
    return int(formed)


def delete(retract_ax, retract_de, vac_ax, vac_de, seed, step, syn: Synapses):
    """Deletion pass in place; returns the number of synapses broken."""
    n = vac_ax.shape[0]
    ra, rd = _c(retract_ax, np.int32), _c(retract_de, np.int32)
    cnt = ctypes.c_int64(syn.count)
    broken = lib().orc_delete(n, _p(ra), _p(rd), _p(vac_ax), _p(vac_de), seed, step,
                              ctypes.byref(cnt), _p(syn.src), _p(syn.tgt), _p(syn.sign))
    syn.count = cnt.value
    return int(broken)


def deliver_spikes(n, syn: Synapses, spiked):
    spiked = _c(spiked, np.uint8)
    out = np.zeros(n, np.int32)
    lib().orc_deliver_spikes(n, syn.count, _p(syn.src), _p(syn.tgt), _p(syn.sign), _p(spiked),
                             _p(out))
    return out


def deliver_rates(n, syn: Synapses, rate, seed, step):
    """Firing-rate delivery (Sec. IV-B): Bernoulli(rate[s]) per (s, t, step)."""
    rate = _c(rate, np.float32)
    out = np.zeros(n, np.int32)
    lib().orc_deliver_rates(n, syn.count, _p(syn.src), _p(syn.tgt), _p(syn.sign), _p(rate),
                            seed, step, _p(out))
    return out


# ------------------------------------------------------- whole update (small)
def update_connectivity(tree: Tree, vac_ax, vac_de, type_, sigma, theta, seed, step,
                        syn: Synapses, threads=1):
    """Reduce, search every vacant axonal element, accept, apply (in place).

    Returns a dict with the request list (canonical query order), accept flags,
    the per-search diagnostics and the number formed.
    """
    tree.reduce(vac_de)
    qi, qe = queries(vac_ax)
    tgt, diag = tree.search_batch(sigma, theta, seed, step, qi, qe, threads=threads)
    acc = accept(tree.n, qi, qe, tgt, vac_de, seed, step)
    formed = apply(qi, tgt, acc, type_, vac_ax, vac_de, syn)
    return {"src": qi, "elem": qe, "tgt": tgt, "accept": acc, "diag": diag, "formed": formed}


def update_connectivity_batch(trees, offsets, vac_ax, vac_de, type_, sigmas, theta, seed, step,
                              syn: Synapses, threads=1):
    """Batched form: independent networks, network b = global ids offsets[b] ..
    offsets[b + 1] - 1 with its own tree (built with id_base = offsets[b]) and sigma.
    Each network searches only its own tree (Sec. III-B per network); the requests of
    all networks then go through one acceptance and one apply over the global ids,
    which equals doing them network by network since no request crosses networks.

    Same return dict as update_connectivity, requests in global canonical order.
    """
    offsets = np.asarray(offsets, np.int64)
    qi_all, qe_all, tgt_all, diag_all = [], [], [], []
    for b, tree in enumerate(trees):
        lo, hi = int(offsets[b]), int(offsets[b + 1])
        assert tree.n == hi - lo and tree.id_base == lo
        tree.reduce(vac_de[lo:hi])
        qi, qe = queries(vac_ax[lo:hi])
        tgt, diag = tree.search_batch(float(sigmas[b]), theta, seed, step, qi, qe,
                                      threads=threads)
        qi_all.append(qi.astype(np.int64) + lo)
        qe_all.append(qe)
        tgt_all.append(np.where(tgt >= 0, tgt.astype(np.int64) + lo, -1))
        diag_all.append(diag)
    qi = np.concatenate(qi_all).astype(np.int32)
    qe = np.concatenate(qe_all).astype(np.int32)
    tgt = np.concatenate(tgt_all).astype(np.int32)
    diag = np.concatenate(diag_all)
    n = int(offsets[-1])
    acc = accept(n, qi, qe, tgt, vac_de, seed, step)
    formed = apply(qi, tgt, acc, type_, vac_ax, vac_de, syn)
    return {"src": qi, "elem": qe, "tgt": tgt, "accept": acc, "diag": diag, "formed": formed}


def mean_length(tree: Tree, sigma, theta, vac_ax, vac_de, grad=True, threads=1):
    """Differentiable form: L = sum_i m_i l_i / sum_i m_i, l_i the attraction-weighted
    mean distance from source i to the centroids of its root frontier (m = vac_ax).
    The tree must have been reduced with the same vac_de. Returns a dict with
    mean, ell (per neuron, NaN when excluded), margin_ac (per neuron: the smallest
    relative distance of a root-frontier criterion test from its tie, inf when none)
    and, with grad, dsigma, the position gradient g (n x 3) and g_abs (n x 3), the same
    sums over the magnitudes of their terms (the scale of their rounding error)."""
    va = _c(vac_ax, np.int32)
    vd = _c(vac_de, np.int32)
    n = tree.n
    ell = np.zeros(n, np.float64)
    ds = np.zeros(1, np.float64)
    g = [np.zeros(n, np.float64) for _ in range(3)] if grad else [None] * 3
    ga = [np.zeros(n, np.float64) for _ in range(3)] if grad else [None] * 3
    margin = np.zeros(n, np.float64)
    m = lib().orc_mean_length(tree._h, float(sigma), float(theta), _p(va), _p(vd), _p(ell),
                              _p(ds), *(_p(a) for a in g), _p(margin), *(_p(a) for a in ga),
                              int(threads))
    out = {"mean": float(m), "ell": ell, "dsigma": float(ds[0]), "margin_ac": margin}
    if grad:
        out["g"] = np.stack(g, 1)
        out["g_abs"] = np.stack(ga, 1)
    return out


def update_connectivity_typed(tree: Tree, vac_ax, vac_de_exc, vac_de_inh, type_, sigma, theta,
                              seed, step, syn: Synapses, threads=1):
    """Typed dendrite pools (reading R16): each neuron has vacant excitatory and
    inhibitory dendritic elements; the tree holds two pools (counts and centroids
    per pool), an excitatory axon (type 0) searches the excitatory pool and an
    inhibitory axon the inhibitory one, and each pool of a target accepts only the
    requests made to it. The two pools never interact, so the update is the plain
    update of Sec. III-A/III-B once per pool, restricted to that pool's axons, with
    the same Philox counters. Updates vac_ax and both pools in place; returns
    {"exc": ..., "inh": ...}, each the dict of update_connectivity for that pool."""
    type_ = np.asarray(type_, np.uint8)
    out = {}
    for kind, name, vde in ((0, "exc", vac_de_exc), (1, "inh", vac_de_inh)):
        va = np.where(type_ == kind, vac_ax, 0).astype(np.int32)
        out[name] = update_connectivity(tree, va, vde, type_, sigma, theta, seed, step, syn,
                                        threads=threads)
        vac_ax[type_ == kind] = va[type_ == kind]
    return out
