"""CPU oracle for the trajectory distance threshold search -- TEST INFRASTRUCTURE ONLY.

Plain FP64 C (``ts_oracle.c``) behind ctypes. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product library never does. The
oracle and the CUDA path share no code. ``ts_rtree.c`` (class ``RTree``) is the CPU R-tree
baseline of the benchmark, built into the same library and using the oracle's pair test.

Every function cites the passage of the paper it follows (Gowanlock & Casanova, Sec. 3.1 problem
definition, Sec. 4.1 flatly structured grid, Sec. 4.2 temporal index, Sec. 4.3 spatiotemporal
index). All functions are pinned by tests in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ts_oracle.c")
_SOURCES = [_SRC, os.path.join(_HERE, "ts_rtree.c"), os.path.join(_HERE, "ts_oracle.h")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libts_oracle.so")
_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE FP64, no contraction, OpenMP for the counting
    baseline). Returns the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SOURCES)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, _SOURCES[1], "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_eval_pairs.argtypes = [_P, _P, _I64, _P, _P, _D, _D, _D, _P, _P, _P, _P]
            lib.orc_eval_pairs.restype = None
            lib.orc_search.argtypes = [_I64, _P, _I64, _P, _D, _D, _D, _I64, _P, _P, _P, _P, _P, _P]
            lib.orc_search.restype = _I64
            lib.orc_search_count.argtypes = [_I64, _P, _I64, _P, _D, _D, _D, _I32, _P, _P]
            lib.orc_search_count.restype = _I64
            lib.orc_search_mt.argtypes = [_I64, _P, _I64, _P, _D, _D, _D, _I32, _P, _I32, _P, _P,
                                          _P, _P, _P, _P]
            lib.orc_search_mt.restype = _I64
            lib.orc_rtree_build.argtypes = [_I64, _P, _I32]
            lib.orc_rtree_build.restype = _P
            lib.orc_rtree_free.argtypes = [_P]
            lib.orc_rtree_free.restype = None
            lib.orc_rtree_shape.argtypes = [_P, _P, _P]
            lib.orc_rtree_shape.restype = None
            lib.orc_rtree_count.argtypes = [_P, _I64, _P, _D, _D, _D, _I32, _P, _P]
            lib.orc_rtree_count.restype = _I64
            lib.orc_rtree_search.argtypes = [_P, _I64, _P, _D, _D, _D, _I32, _I64, _P, _P, _P,
                                             _P]
            lib.orc_rtree_search.restype = _I64
            lib.orc_openmp_max_threads.argtypes = []
            lib.orc_openmp_max_threads.restype = _I32
            lib.orc_temporal_index.argtypes = [_I64, _P, _P, _I32, _P, _P, _P, _P, _P, _P, _P]
            lib.orc_temporal_index.restype = ctypes.c_int
            lib.orc_temporal_schedule.argtypes = [_I32, _P, _P, _P, _I64, _P, _P, _P, _P]
            lib.orc_temporal_schedule.restype = None
            lib.orc_st_params.argtypes = [_I64, _P, _P, _I32, _P, _P, _P]
            lib.orc_st_params.restype = None
            lib.orc_st_dim.argtypes = [_I64, _P, _P, _P, _I32, _D, _D, _I32, _I64, _P, _P]
            lib.orc_st_dim.restype = _I64
            lib.orc_st_schedule.argtypes = [_I32, _P, _P, _P, _P, _P, _P, _P, _I64, _P, _P, _P,
                                            _P, _D, _P, _P, _P]
            lib.orc_st_schedule.restype = None
            lib.orc_grid_params.argtypes = [_I64, _P, _P, _I32, _P, _P]
            lib.orc_grid_params.restype = None
            lib.orc_fsg.argtypes = [_I64, _P, _P, _I32, _P, _P, _I64, _P, _P]
            lib.orc_fsg.restype = _I64
            lib.orc_fsg_candidates.argtypes = [_I64, _P, _P, _I32, _P, _P, _P, _P, _I64, _P, _P,
                                               _D, _P, _P]
            lib.orc_fsg_candidates.restype = None
            lib.orc_grid1.argtypes = [_I64, _P, _I32, _P, _P, _P, _P]
            lib.orc_grid1.restype = _I64
            lib.orc_grid1_candidates.argtypes = [_I32, _P, _P, _P, _P, _I64, _P, _P, _P, _P, _D,
                                                 _P, _P]
            lib.orc_grid1_candidates.restype = None
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class _Cols:
    """Keeps 8 contiguous FP64 columns alive and exposes them as a C array of pointers."""

    def __init__(self, cols):
        self.cols = [_f64(c) for c in cols]
        if len(self.cols) != 8:
            raise ValueError("a segment set has 8 columns: x0 y0 z0 t0 x1 y1 z1 t1")
        self.n = int(self.cols[0].shape[0])
        self.arr = (ctypes.c_void_p * 8)(*[c.ctypes.data for c in self.cols])

    @property
    def ptr(self):
        return ctypes.cast(self.arr, ctypes.c_void_p)


def _cols(segs):
    if hasattr(segs, "arrays"):
        return _Cols(segs.arrays())
    return _Cols(segs)


def eval_pairs(db, queries, qi, ei, t_start, t_end, d):
    """Evaluate explicit (query, entry) pairs with the interaction test (Sec. 3.1). Returns
    (hit bool array, t_in, t_out, s_min)."""
    lib = _load()
    e, q = _cols(db), _cols(queries)
    qi = np.ascontiguousarray(qi, dtype=np.int64)
    ei = np.ascontiguousarray(ei, dtype=np.int64)
    n = qi.shape[0]
    hit = np.zeros(n, dtype=np.int32)
    tin, tout, smin = (np.empty(n) for _ in range(3))
    lib.orc_eval_pairs(e.ptr, q.ptr, n, _ptr(qi), _ptr(ei), t_start, t_end, d, _ptr(hit),
                       _ptr(tin), _ptr(tout), _ptr(smin))
    return hit.astype(bool), tin, tout, smin


def search(db, queries, t_start, t_end, d, threads=None):
    """All-pairs distance threshold search (Sec. 3.1) with exact temporal pruning, on `threads`
    OpenMP threads (all by default; 1 = the single-threaded loop). Returns a dict of arrays
    q_idx, e_idx, t_in, t_out, s_min sorted by (q_idx, e_idx), and n_tests."""
    lib = _load()
    if threads is None:
        threads = max_threads()
    if threads > 1:
        e, q = _cols(db), _cols(queries)
        cnt = np.zeros(max(q.n, 1), dtype=np.int64)
        ntests = np.zeros(1, dtype=np.int64)
        total = lib.orc_search_mt(e.n, e.ptr, q.n, q.ptr, t_start, t_end, d, int(threads),
                                  _ptr(cnt), 0, None, None, None, None, None, _ptr(ntests))
        if total < 0:
            raise MemoryError("oracle allocation failed")
        oq = np.empty(total, dtype=np.uint32)
        oe = np.empty(total, dtype=np.uint32)
        tin, tout, smin = (np.empty(total) for _ in range(3))
        if total:
            got = lib.orc_search_mt(e.n, e.ptr, q.n, q.ptr, t_start, t_end, d, int(threads),
                                    _ptr(cnt), 1, _ptr(oq), _ptr(oe), _ptr(tin), _ptr(tout),
                                    _ptr(smin), None)
            if got != total:
                raise RuntimeError("oracle: the two passes disagree")
        order = np.lexsort((oe, oq))
        return {"q_idx": oq[order], "e_idx": oe[order], "t_in": tin[order],
                "t_out": tout[order], "s_min": smin[order], "n_tests": int(ntests[0])}
    e, q = _cols(db), _cols(queries)
    cap = 1 << 16
    while True:
        oq = np.empty(cap, dtype=np.uint32)
        oe = np.empty(cap, dtype=np.uint32)
        tin, tout, smin = (np.empty(cap) for _ in range(3))
        ntests = np.zeros(1, dtype=np.int64)
        cnt = lib.orc_search(e.n, e.ptr, q.n, q.ptr, t_start, t_end, d, cap, _ptr(oq), _ptr(oe),
                             _ptr(tin), _ptr(tout), _ptr(smin), _ptr(ntests))
        if cnt < 0:
            raise MemoryError("oracle allocation failed")
        if cnt <= cap:
            break
        cap = int(cnt)
    order = np.lexsort((oe[:cnt], oq[:cnt]))
    return {"q_idx": oq[:cnt][order], "e_idx": oe[:cnt][order], "t_in": tin[:cnt][order],
            "t_out": tout[:cnt][order], "s_min": smin[:cnt][order], "n_tests": int(ntests[0])}


def search_count(db, queries, t_start, t_end, d, threads=1):
    """Hit count of the same search on `threads` OpenMP threads. Returns (hits, tests, qsegs)."""
    lib = _load()
    e, q = _cols(db), _cols(queries)
    nt = np.zeros(1, dtype=np.int64)
    nqs = np.zeros(1, dtype=np.int64)
    cnt = lib.orc_search_count(e.n, e.ptr, q.n, q.ptr, t_start, t_end, d, int(threads), _ptr(nt),
                               _ptr(nqs))
    if cnt < 0:
        raise MemoryError("oracle allocation failed")
    return int(cnt), int(nt[0]), int(nqs[0])


def max_threads() -> int:
    return int(_load().orc_openmp_max_threads())


def temporal_index(t0, t1, m):
    """Temporal index of Sec. 4.2. Returns dict perm (sorted position -> original index), bin_of
    (per sorted position), bin_start, bin_end, bin_off (m+1), tmin, b."""
    lib = _load()
    t0, t1 = _f64(t0), _f64(t1)
    n = t0.shape[0]
    perm = np.empty(n, dtype=np.int64)
    bin_of = np.empty(n, dtype=np.int32)
    bs, be = np.empty(m), np.empty(m)
    off = np.empty(m + 1, dtype=np.int64)
    tmin, b = np.zeros(1), np.zeros(1)
    rc = lib.orc_temporal_index(n, _ptr(t0), _ptr(t1), m, _ptr(perm), _ptr(bin_of), _ptr(bs),
                                _ptr(be), _ptr(off), _ptr(tmin), _ptr(b))
    if rc != 0:
        raise ValueError("temporal index: invalid input")
    return {"perm": perm, "bin_of": bin_of, "bin_start": bs, "bin_end": be, "bin_off": off,
            "tmin": float(tmin[0]), "b": float(b[0])}


def temporal_schedule(tidx, w0, w1):
    """Temporal schedule S of Sec. 4.2: per query window the entry range [lo, hi)."""
    lib = _load()
    w0, w1 = _f64(w0), _f64(w1)
    nq = w0.shape[0]
    lo = np.empty(nq, dtype=np.int64)
    hi = np.empty(nq, dtype=np.int64)
    m = tidx["bin_start"].shape[0]
    lib.orc_temporal_schedule(m, _ptr(tidx["bin_start"]), _ptr(tidx["bin_end"]),
                              _ptr(tidx["bin_off"]), nq, _ptr(w0), _ptr(w1), _ptr(lo), _ptr(hi))
    return lo, hi


def st_params(emin, emax, v):
    """Subbin origin, width and effective count of one dimension (Sec. 4.3)."""
    lib = _load()
    emin, emax = _f64(emin), _f64(emax)
    lo, w = np.zeros(1), np.zeros(1)
    ve = np.zeros(1, dtype=np.int32)
    lib.orc_st_params(emin.shape[0], _ptr(emin), _ptr(emax), int(v), _ptr(lo), _ptr(w), _ptr(ve))
    return float(lo[0]), float(w[0]), int(ve[0])


def st_dim(emin_sorted, emax_sorted, bin_of, m, lo, w, v):
    """One dimension's id array and (j, i) offsets of the spatiotemporal index (Sec. 4.3)."""
    lib = _load()
    emin, emax = _f64(emin_sorted), _f64(emax_sorted)
    bin_of = np.ascontiguousarray(bin_of, dtype=np.int32)
    n = emin.shape[0]
    off = np.empty(v * m + 1, dtype=np.int64)
    cap = 2 * n + 16
    while True:
        ids = np.empty(cap, dtype=np.uint32)
        ln = lib.orc_st_dim(n, _ptr(emin), _ptr(emax), _ptr(bin_of), m, lo, w, v, cap, _ptr(ids),
                            _ptr(off))
        if ln <= cap:
            return ids[:ln], off
        cap = int(ln)


def st_schedule(tidx, dims, qmin, qmax, w0, w1, d):
    """Spatiotemporal schedule of Sec. 4.3. dims: list of 3 dicts with lo, w, v, off.
    Returns (sel, lo, hi)."""
    lib = _load()
    m = tidx["bin_start"].shape[0]
    sub_lo = np.array([x["lo"] for x in dims], dtype=np.float64)
    sub_w = np.array([x["w"] for x in dims], dtype=np.float64)
    sub_v = np.array([x["v"] for x in dims], dtype=np.int32)
    offs = [np.ascontiguousarray(x["off"], dtype=np.int64) for x in dims]
    off_arr = (ctypes.c_void_p * 3)(*[o.ctypes.data for o in offs])
    qmin = [_f64(a) for a in qmin]
    qmax = [_f64(a) for a in qmax]
    qmin_arr = (ctypes.c_void_p * 3)(*[a.ctypes.data for a in qmin])
    qmax_arr = (ctypes.c_void_p * 3)(*[a.ctypes.data for a in qmax])
    w0, w1 = _f64(w0), _f64(w1)
    nq = w0.shape[0]
    sel = np.empty(nq, dtype=np.int32)
    lo = np.empty(nq, dtype=np.int64)
    hi = np.empty(nq, dtype=np.int64)
    lib.orc_st_schedule(m, _ptr(tidx["bin_start"]), _ptr(tidx["bin_end"]), _ptr(tidx["bin_off"]),
                        _ptr(sub_lo), _ptr(sub_w), _ptr(sub_v), ctypes.cast(off_arr, _P), nq,
                        ctypes.cast(qmin_arr, _P), ctypes.cast(qmax_arr, _P), _ptr(w0), _ptr(w1),
                        d, _ptr(sel), _ptr(lo), _ptr(hi))
    return sel, lo, hi


def grid_params(emin, emax, g):
    """Grid origin and cell width of one dimension for the flatly structured grid (Sec. 4.1)."""
    lib = _load()
    emin, emax = _f64(emin), _f64(emax)
    lo, w = np.zeros(1), np.zeros(1)
    lib.orc_grid_params(emin.shape[0], _ptr(emin), _ptr(emax), int(g), _ptr(lo), _ptr(w))
    return float(lo[0]), float(w[0])


def fsg(emin3, emax3, g, lo3, w3):
    """Flatly structured grid of Sec. 4.1: lookup array A and per-cell offsets (g^3 + 1)."""
    lib = _load()
    emin = [_f64(a) for a in emin3]
    emax = [_f64(a) for a in emax3]
    n = emin[0].shape[0]
    ea = (ctypes.c_void_p * 3)(*[a.ctypes.data for a in emin])
    eb = (ctypes.c_void_p * 3)(*[a.ctypes.data for a in emax])
    lo = _f64(lo3)
    w = _f64(w3)
    off = np.empty(g * g * g + 1, dtype=np.int64)
    cap = 4 * n + 16
    while True:
        A = np.empty(cap, dtype=np.uint32)
        ln = lib.orc_fsg(n, ctypes.cast(ea, _P), ctypes.cast(eb, _P), g, _ptr(lo), _ptr(w), cap,
                         _ptr(A), _ptr(off))
        if ln < 0:
            raise MemoryError("oracle allocation failed")
        if ln <= cap:
            return A[:ln], off
        cap = int(ln)


def fsg_candidates(emin3, emax3, g, lo3, w3, A, off, qmin3, qmax3, d):
    """Per-query candidate counts of the spatial index (Sec. 4.1): (raw, duplicate-free)."""
    lib = _load()
    emin = [_f64(a) for a in emin3]
    emax = [_f64(a) for a in emax3]
    ea = (ctypes.c_void_p * 3)(*[a.ctypes.data for a in emin])
    eb = (ctypes.c_void_p * 3)(*[a.ctypes.data for a in emax])
    qmin = [_f64(a) for a in qmin3]
    qmax = [_f64(a) for a in qmax3]
    qa = (ctypes.c_void_p * 3)(*[a.ctypes.data for a in qmin])
    qb = (ctypes.c_void_p * 3)(*[a.ctypes.data for a in qmax])
    lo, w = _f64(lo3), _f64(w3)
    A = np.ascontiguousarray(A, dtype=np.uint32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    nq = qmin[0].shape[0]
    raw = np.empty(nq, dtype=np.int64)
    uniq = np.empty(nq, dtype=np.int64)
    lib.orc_fsg_candidates(emin[0].shape[0], ctypes.cast(ea, _P), ctypes.cast(eb, _P), g,
                           _ptr(lo), _ptr(w), _ptr(A), _ptr(off), nq, ctypes.cast(qa, _P),
                           ctypes.cast(qb, _P), d, _ptr(raw), _ptr(uniq))
    return raw, uniq


def grid1(emin3, g, lo3, w3):
    """One-cell-per-entry grid (Sec. 4.1 grid, entries keyed by their MBB minimum corner):
    lookup array A and per-cell offsets (g^3 + 1)."""
    lib = _load()
    emin = [_f64(a) for a in emin3]
    n = emin[0].shape[0]
    ea = (ctypes.c_void_p * 3)(*[a.ctypes.data for a in emin])
    lo, w = _f64(lo3), _f64(w3)
    off = np.empty(g * g * g + 1, dtype=np.int64)
    A = np.empty(max(n, 1), dtype=np.uint32)
    ln = lib.orc_grid1(n, ctypes.cast(ea, _P), g, _ptr(lo), _ptr(w), _ptr(A), _ptr(off))
    if ln < 0:
        raise MemoryError("oracle allocation failed")
    return A[:n], off


def grid1_candidates(g, lo3, w3, longest3, off, qmin3, qmax3, w0, w1, d):
    """Per query: (number of z-runs, number of candidates) in the one-cell-per-entry grid."""
    lib = _load()
    qmin = [_f64(a) for a in qmin3]
    qmax = [_f64(a) for a in qmax3]
    qa = (ctypes.c_void_p * 3)(*[a.ctypes.data for a in qmin])
    qb = (ctypes.c_void_p * 3)(*[a.ctypes.data for a in qmax])
    lo, w, L = _f64(lo3), _f64(w3), _f64(longest3)
    off = np.ascontiguousarray(off, dtype=np.int64)
    w0, w1 = _f64(w0), _f64(w1)
    nq = w0.shape[0]
    runs = np.empty(nq, dtype=np.int64)
    cand = np.empty(nq, dtype=np.int64)
    lib.orc_grid1_candidates(g, _ptr(lo), _ptr(w), _ptr(L), _ptr(off), nq, ctypes.cast(qa, _P),
                             ctypes.cast(qb, _P), _ptr(w0), _ptr(w1), d, _ptr(runs), _ptr(cand))
    return runs, cand


class RTree:
    """CPU in-memory R-tree over a database (the paper's CPU comparator, Sec. 5): groups of r
    consecutive segments of a trajectory, one 4-D box per group, bulk-loaded (STR packing);
    queries on OpenMP threads test the segments of every group whose box meets the query's
    window and d-widened MBB with the oracle's interaction test. Keeps the database columns
    alive while it lives."""

    def __init__(self, db, r=1):
        lib = _load()
        self._cols = _cols(db)
        self.r = int(r)
        self._h = lib.orc_rtree_build(self._cols.n, self._cols.ptr, self.r)
        if not self._h:
            raise MemoryError("R-tree build failed")

    def shape(self):
        ng, nl = np.zeros(1, dtype=np.int64), np.zeros(1, dtype=np.int32)
        _load().orc_rtree_shape(self._h, _ptr(ng), _ptr(nl))
        return int(ng[0]), int(nl[0])

    def count(self, queries, t_start, t_end, d, threads=None):
        """(hits, interaction tests, query segments) on `threads` threads (all by default)."""
        q = _cols(queries)
        nt, nq = np.zeros(1, dtype=np.int64), np.zeros(1, dtype=np.int64)
        threads = max_threads() if threads is None else int(threads)
        c = _load().orc_rtree_count(self._h, q.n, q.ptr, t_start, t_end, d, threads, _ptr(nt),
                                    _ptr(nq))
        return int(c), int(nt[0]), int(nq[0])

    def search(self, queries, t_start, t_end, d, threads=None):
        """Every hit as arrays q_idx, e_idx, t_in, t_out sorted by (q_idx, e_idx)."""
        lib = _load()
        q = _cols(queries)
        threads = max_threads() if threads is None else int(threads)
        cap = 1 << 16
        while True:
            oq, oe = np.empty(cap, dtype=np.int64), np.empty(cap, dtype=np.int64)
            ti, to = np.empty(cap), np.empty(cap)
            n = lib.orc_rtree_search(self._h, q.n, q.ptr, t_start, t_end, d, threads, cap,
                                     _ptr(oq), _ptr(oe), _ptr(ti), _ptr(to))
            if n < 0:
                raise MemoryError("R-tree search failed")
            if n <= cap:
                break
            cap = int(n)
        order = np.lexsort((oe[:n], oq[:n]))
        return {"q_idx": oq[:n][order].astype(np.uint32), "e_idx": oe[:n][order].astype(np.uint32),
                "t_in": ti[:n][order], "t_out": to[:n][order]}

    def free(self):
        if self._h:
            _load().orc_rtree_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
