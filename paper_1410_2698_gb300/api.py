"""Python binding of the C ABI (include/ts.h): same names, argument marshalling only.

Segment sets may be given as a ``workloads.Segments`` of numpy arrays (host memory: the library
copies them to the device inside the call) or as any object whose eight fields x0, y0, z0, t0,
x1, y1, z1, t1 are contiguous float64 CUDA tensors (device memory, read in place). Every step of
the search runs in the CUDA library; nothing here computes.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import TsError, check

FIELDS8 = ("x0", "y0", "z0", "t0", "x1", "y1", "z1", "t1")


def _current_stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:  # pragma: no cover
        pass
    return ctypes.c_void_p(0)


def _columns(segs):
    if isinstance(segs, dict):
        return [segs[f] for f in FIELDS8]
    if isinstance(segs, (list, tuple)) and len(segs) == 8:
        return list(segs)
    return [getattr(segs, f) for f in FIELDS8]


def make_segments(segs):
    """Marshal a segment set into a ts_segments struct. Returns (struct, keepalive)."""
    cols = _columns(segs)
    first = cols[0]
    s = _lib.ts_segments()
    keep = []
    if isinstance(first, np.ndarray):
        arrs = [np.ascontiguousarray(c, dtype=np.float64) for c in cols]
        n = arrs[0].shape[0]
        for name, a in zip(FIELDS8, arrs):
            if a.shape != (n,):
                raise ValueError("all eight columns must be 1-D of equal length")
            setattr(s, name, a.ctypes.data if n else None)
        s.n = n
        s.on_host = 1
        keep = arrs
    else:  # torch tensors: on the GPU, or in (pinned) host memory
        import torch
        n = int(first.shape[0])
        on_gpu = bool(first.is_cuda)
        for name, t in zip(FIELDS8, cols):
            if not (isinstance(t, torch.Tensor) and bool(t.is_cuda) == on_gpu
                    and t.dtype == torch.float64 and t.is_contiguous() and t.dim() == 1
                    and int(t.shape[0]) == n):
                raise ValueError("tensor columns must be contiguous 1-D float64 tensors, all on "
                                 "the GPU or all on the host")
            setattr(s, name, t.data_ptr() if n else None)
        s.n = n
        s.on_host = 0 if on_gpu else 1
        keep = cols
    return s, keep


class Index:
    """Owner of a ts_index handle."""

    def __init__(self, handle, n):
        self._h = handle
        self.n = n

    @property
    def handle(self):
        return self._h

    def info(self):
        return ts_index_get_info(self)

    def free(self):
        if self._h:
            _lib.load().ts_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Result:
    """Owner of a ts_result handle."""

    def __init__(self, handle, status):
        self._h = handle
        self.status = status

    @property
    def handle(self):
        return self._h

    @property
    def count(self) -> int:
        return int(_lib.load().ts_result_count(self._h))

    @property
    def stats(self) -> dict:
        return ts_result_stats(self)

    def to_host(self, stream=None, sort=False):
        return ts_result_copy_to_host(self, stream=stream, sort=sort)

    def device_arrays(self):
        return ts_result_arrays(self)

    def free(self):
        if self._h:
            _lib.load().ts_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def ts_version() -> str:
    return _lib.load().ts_version().decode()


def ts_build_index(db, kind="temporal", t_bins=0, sub_bins=0, grid_cells=0, stream=None) -> Index:
    lib = _lib.load()
    s, keep = make_segments(db)
    p = _lib.ts_index_params(_lib.KINDS[kind] if isinstance(kind, str) else int(kind),
                             int(t_bins), int(sub_bins), int(grid_cells))
    out = ctypes.c_void_p()
    check(lib.ts_build_index(ctypes.byref(s), ctypes.byref(p), _current_stream(stream),
                             ctypes.byref(out)))
    del keep
    return Index(out, int(s.n))


def ts_index_get_info(index: Index) -> dict:
    lib = _lib.load()
    info = _lib.ts_index_info()
    check(lib.ts_index_get_info(index.handle, ctypes.byref(info)))
    return info.as_dict()


def ts_index_export(index: Index, field: str, dim: int = 0) -> np.ndarray:
    lib = _lib.load()
    fid = _lib.FIELDS[field]
    size = ctypes.c_uint64(0)
    st = lib.ts_index_export(index.handle, fid, dim, None, 0, ctypes.byref(size))
    if st not in (_lib.TS_OK, 4):
        check(st)
    dtype = np.float64 if field in ("bin_start", "bin_end") else np.uint32
    out = np.empty(int(size.value) // np.dtype(dtype).itemsize, dtype=dtype)
    check(lib.ts_index_export(index.handle, fid, dim, out.ctypes.data if out.size else None,
                              int(size.value), ctypes.byref(size)))
    return out


def _qparams(d, t_start, t_end, max_results):
    return _lib.ts_query_params(float(d), float(t_start), float(t_end), int(max_results))


def ts_schedule(index: Index, queries, d, t_start, t_end, stream=None):
    lib = _lib.load()
    s, keep = make_segments(queries)
    n = int(s.n)
    sel = np.zeros(n, dtype=np.int32)
    lo = np.zeros(n, dtype=np.uint64)
    hi = np.zeros(n, dtype=np.uint64)
    qp = _qparams(d, t_start, t_end, 0)
    check(lib.ts_schedule(index.handle, ctypes.byref(s), ctypes.byref(qp), _current_stream(stream),
                          sel.ctypes.data, lo.ctypes.data, hi.ctypes.data))
    del keep
    return sel, lo, hi


def ts_search(index: Index, queries, d, t_start, t_end, max_results=0, stream=None) -> Result:
    """Search; raises TsError on failure. With max_results exceeded the returned Result has
    status TS_ERR_CAPACITY (4), the exact count and no rows."""
    lib = _lib.load()
    s, keep = make_segments(queries)
    qp = _qparams(d, t_start, t_end, max_results)
    out = ctypes.c_void_p()
    st = lib.ts_search(index.handle, ctypes.byref(s), ctypes.byref(qp), _current_stream(stream),
                       ctypes.byref(out))
    del keep
    if st == 4 and out.value:
        return Result(out, st)
    check(st)
    return Result(out, st)


def ts_search_points(index: Index, x, y, z, d, t_start, t_end, max_results=0,
                     stream=None) -> Result:
    """Stationary-point search: every database segment within d of a point (x[i], y[i], z[i]) at
    some instant of [t_start, t_end]. x, y, z: numpy arrays (host) or CUDA tensors (device)."""
    lib = _lib.load()
    on_host = isinstance(x, np.ndarray)
    if on_host:
        cols = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z)]
        ptrs = [c.ctypes.data for c in cols]
    else:
        cols = [a.contiguous() for a in (x, y, z)]
        ptrs = [c.data_ptr() for c in cols]
    n = int(cols[0].shape[0])
    if any(int(c.shape[0]) != n for c in cols):
        raise ValueError("x, y and z must have the same length")
    qp = _qparams(d, t_start, t_end, max_results)
    out = ctypes.c_void_p()
    st = lib.ts_search_points(index.handle, ctypes.c_void_p(ptrs[0]), ctypes.c_void_p(ptrs[1]),
                              ctypes.c_void_p(ptrs[2]), n, int(on_host), ctypes.byref(qp),
                              _current_stream(stream), ctypes.byref(out))
    del cols
    if st == 4 and out.value:
        return Result(out, st)
    check(st)
    return Result(out, st)


def ts_result_count(result: Result) -> int:
    return result.count


def ts_result_stats(result: Result) -> dict:
    lib = _lib.load()
    st = _lib.ts_search_stats()
    check(lib.ts_result_stats(result.handle, ctypes.byref(st)))
    return st.as_dict()


def ts_result_arrays(result: Result):
    """Device pointers (ints) of q_idx, e_idx, t_in, t_out."""
    lib = _lib.load()
    ptrs = [ctypes.c_void_p() for _ in range(4)]
    check(lib.ts_result_arrays(result.handle, *[ctypes.byref(p) for p in ptrs]))
    return tuple(p.value for p in ptrs)


def ts_result_copy_to_host(result: Result, stream=None, sort=False) -> dict:
    lib = _lib.load()
    n = result.count
    q = np.empty(n, dtype=np.uint32)
    e = np.empty(n, dtype=np.uint32)
    tin = np.empty(n, dtype=np.float64)
    tout = np.empty(n, dtype=np.float64)
    if n:
        check(lib.ts_result_copy_to_host(result.handle, q.ctypes.data, e.ctypes.data,
                                         tin.ctypes.data, tout.ctypes.data,
                                         _current_stream(stream)))
    out = {"q_idx": q, "e_idx": e, "t_in": tin, "t_out": tout}
    if sort and n:
        order = np.lexsort((e, q))
        out = {k: v[order] for k, v in out.items()}
    return out


def ts_free(obj):
    obj.free()


def ts_search_brute_noalloc(db, queries, d, t_start, t_end, q_idx, e_idx, t_in, t_out,
                            stream=None):
    """All-pairs search into caller-provided device arrays, without any allocation by the
    library (for callers that cannot allocate device memory). db and queries: eight float64 CUDA
    tensors each; q_idx, e_idx (int32/uint32) and t_in, t_out (float64): CUDA tensors of equal
    length (the capacity). Returns (status, row count); status 4 (capacity) writes no rows."""
    lib = _lib.load()
    s_db, keep1 = make_segments(db)
    s_q, keep2 = make_segments(queries)
    if s_db.on_host or s_q.on_host:
        raise ValueError("the no-allocation search takes device tensors only")
    cap = int(q_idx.shape[0])
    for t in (e_idx, t_in, t_out):
        if int(t.shape[0]) != cap:
            raise ValueError("output arrays must have equal length")
    qp = _qparams(d, t_start, t_end, 0)
    count = ctypes.c_uint64(0)
    st = lib.ts_search_brute_noalloc(ctypes.byref(s_db), ctypes.byref(s_q), ctypes.byref(qp),
                                     q_idx.data_ptr(), e_idx.data_ptr(), t_in.data_ptr(),
                                     t_out.data_ptr(), cap, ctypes.byref(count),
                                     _current_stream(stream))
    del keep1, keep2
    if st not in (_lib.TS_OK, 4):
        check(st)
    return st, int(count.value)


def ts_measure_alu_peaks() -> dict:
    """Measured FP32 and FP64 FMA throughput of the current device (TFLOP/s)."""
    lib = _lib.load()
    a, b = ctypes.c_double(), ctypes.c_double()
    check(lib.ts_measure_alu_peaks(ctypes.byref(a), ctypes.byref(b)))
    return {"fp32_tflops": a.value, "fp64_tflops": b.value}


def ts_eval_refined_estimates(x) -> dict:
    """The exact test's refined 1/x and sqrt(x) and the CUDA runtime's, for a host array x."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = {k: np.empty_like(x) for k in ("rcp_est", "sqrt_est", "rcp_ref", "sqrt_ref")}
    check(_lib.load().ts_eval_refined_estimates(
        x.ctypes.data, x.size, *(out[k].ctypes.data for k in ("rcp_est", "sqrt_est", "rcp_ref",
                                                               "sqrt_ref"))))
    return out


def ts_debug_inject_stall(limit_ns: int) -> None:
    """Test hook: the next plain search's count pass times out after limit_ns (TS_ERR_TIMEOUT)."""
    check(_lib.load().ts_debug_inject_stall(int(limit_ns)))


def ts_kernel_launches() -> int:
    return int(_lib.load().ts_kernel_launches())


def ts_last_error() -> str:
    return _lib.load().ts_last_error().decode()


# ---------------------------------------------------------------------------------------------
# batched search
# ---------------------------------------------------------------------------------------------
def _requests(requests):
    """requests: list of (queries, d, t_start, t_end) or (queries, d, t_start, t_end, max_results).
    Returns ctypes arrays of ts_segments and ts_query_params and the keep-alive list."""
    n = len(requests)
    segs = (_lib.ts_segments * n)()
    qps = (_lib.ts_query_params * n)()
    keep = []
    for r, req in enumerate(requests):
        q, d, ts, te = req[:4]
        mr = req[4] if len(req) > 4 else 0
        s, k = make_segments(q)
        segs[r] = s
        keep.append(k)
        qps[r] = _qparams(d, ts, te, mr)
    return segs, qps, keep


class PreparedRequests:
    """Requests marshalled once for repeated BatchPlan.run calls (the request table is built
    from the columns' addresses: the columns must stay alive and in place while it is used)."""

    def __init__(self, requests):
        self.n = len(requests)
        self.segs, self.qps, self._keep = _requests(requests)
        self._requests = list(requests)


def prepare_requests(requests) -> PreparedRequests:
    return PreparedRequests(requests)


def ts_search_batch(index: Index, requests, stream=None):
    """One pipeline for many requests; returns one Result per request."""
    lib = _lib.load()
    segs, qps, keep = _requests(requests)
    n = len(requests)
    outs = (ctypes.c_void_p * n)()
    st = lib.ts_search_batch(index.handle, n, segs, qps, _current_stream(stream), outs)
    del keep
    if st not in (_lib.TS_OK, 4):
        check(st)
    return [Result(ctypes.c_void_p(outs[r]), st) for r in range(n)]


class _Outcome(dict):
    """A batch run's outcome; its "stats" entry is converted from the C struct on first use."""

    def __init__(self, st):
        super().__init__(rows=int(st.rows), nreq=int(st.nreq), overflow=bool(st.overflow))
        self._st = st

    def __missing__(self, key):
        if key == "stats":
            v = self._st.stats.as_dict()
            self[key] = v
            return v
        raise KeyError(key)


class BatchPlan:
    """Reusable batched pipeline with fixed capacities (ts_batch_*), optionally replayed as a
    CUDA graph."""

    def __init__(self, index: Index, max_requests, max_queries, max_rows, tile_records=0,
                 use_graph=True, pair_blocks=0, max_units=0, max_tiles=0, stream=None,
                 scratch_rows=0):
        lib = _lib.load()
        p = _lib.ts_batch_params(int(max_requests), int(tile_records), int(max_queries),
                                 int(max_rows), int(max_units), int(max_tiles), int(use_graph),
                                 int(pair_blocks), int(scratch_rows))
        h = ctypes.c_void_p()
        check(lib.ts_batch_create(index.handle, ctypes.byref(p), _current_stream(stream),
                                  ctypes.byref(h)))
        self._h = h
        self.index = index
        self._keep = None

    @property
    def handle(self):
        return self._h

    def run(self, requests, stream=None):
        """Run the plan on a list of requests, or on PreparedRequests (marshalled once)."""
        lib = _lib.load()
        if isinstance(requests, PreparedRequests):
            segs, qps, n = requests.segs, requests.qps, requests.n
            self._keep = requests
        else:
            segs, qps, keep = _requests(requests)
            n = len(requests)
            self._keep = (segs, qps, keep)
        check(lib.ts_batch_run(self._h, n, segs, qps, _current_stream(stream)))

    def wait(self) -> dict:
        """Wait for the last run: {"rows", "nreq", "overflow", "stats"} (the statistics dict is
        built when first read)."""
        lib = _lib.load()
        st = _lib.ts_batch_status()
        check(lib.ts_batch_wait(self._h, ctypes.byref(st)))
        self._keep = None
        self._last = (int(st.nreq), int(st.rows))
        return _Outcome(st)

    def request_rows(self, r):
        lib = _lib.load()
        first, count = ctypes.c_uint64(), ctypes.c_uint64()
        check(lib.ts_batch_request_rows(self._h, r, ctypes.byref(first), ctypes.byref(count)))
        return int(first.value), int(count.value)

    def request_to_host(self, r, sort=False, out=None) -> dict:
        """Copy request r's rows to host arrays: new numpy arrays, or the first rows of `out`
        (a dict of q_idx, e_idx, t_in, t_out arrays, e.g. views of pinned buffers, large
        enough for the rows)."""
        lib = _lib.load()
        first, n = self.request_rows(r)
        if out is not None:
            if any(len(out[k]) < n for k in ("q_idx", "e_idx", "t_in", "t_out")):
                raise ValueError(f"output buffers hold fewer than the request's {n} rows")
            q, e, tin, tout = (out[k][:n] for k in ("q_idx", "e_idx", "t_in", "t_out"))
        else:
            q = np.empty(n, dtype=np.uint32)
            e = np.empty(n, dtype=np.uint32)
            tin = np.empty(n, dtype=np.float64)
            tout = np.empty(n, dtype=np.float64)
        if n:
            check(lib.ts_batch_copy_rows(self._h, first, n, q.ctypes.data, e.ctypes.data,
                                         tin.ctypes.data, tout.ctypes.data))
        out = {"q_idx": q, "e_idx": e, "t_in": tin, "t_out": tout}
        if sort and n:
            order = np.lexsort((e, q))
            out = {k: v[order] for k, v in out.items()}
        return out

    def copy_rows(self, first, count, out):
        """Copy rows [first, first + count) of the last run into the first `count` entries of
        `out` (a dict of q_idx, e_idx, t_in, t_out host arrays, e.g. views of pinned buffers)."""
        if any(len(out[k]) < count for k in ("q_idx", "e_idx", "t_in", "t_out")):
            raise ValueError(f"output buffers hold fewer than {count} rows")
        if count:
            check(_lib.load().ts_batch_copy_rows(
                self._h, int(first), int(count), out["q_idx"].ctypes.data,
                out["e_idx"].ctypes.data, out["t_in"].ctypes.data, out["t_out"].ctypes.data))
        return 24 * int(count)

    def rows_to_host(self, out=None):
        """Copy every row of the last run (requests in order, each request's rows contiguous) to
        host arrays in one call: new numpy arrays or the first rows of `out`. Returns the rows
        and each request's (first, count) within them."""
        nreq, total = getattr(self, "_last", (0, 0))
        spans = [self.request_rows(r) for r in range(nreq)]
        lib = _lib.load()
        if out is not None:
            if any(len(out[k]) < total for k in ("q_idx", "e_idx", "t_in", "t_out")):
                raise ValueError(f"output buffers hold fewer than the run's {total} rows")
            q, e, tin, tout = (out[k][:total] for k in ("q_idx", "e_idx", "t_in", "t_out"))
        else:
            q = np.empty(total, dtype=np.uint32)
            e = np.empty(total, dtype=np.uint32)
            tin = np.empty(total, dtype=np.float64)
            tout = np.empty(total, dtype=np.float64)
        if total:
            check(lib.ts_batch_copy_rows(self._h, 0, total, q.ctypes.data, e.ctypes.data,
                                         tin.ctypes.data, tout.ctypes.data))
        return {"q_idx": q, "e_idx": e, "t_in": tin, "t_out": tout}, spans

    def free(self):
        if self._h:
            _lib.load().ts_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------------------------------------
# served search
# ---------------------------------------------------------------------------------------------
class Server:
    """Request loop on a resident index (ts_server_*): submit from any thread, wait per ticket."""

    def __init__(self, index: Index, max_batch_requests=64, max_batch_queries=1 << 20,
                 max_batch_rows=1 << 26, max_inflight=2, tile_records=0, use_graph=True,
                 linger_us=200, scratch_rows=0, mem_budget_bytes=0, admit_wait_ms=0):
        lib = _lib.load()
        p = _lib.ts_server_params(int(max_inflight), int(max_batch_requests),
                                  int(max_batch_queries), int(max_batch_rows),
                                  int(tile_records), int(use_graph), int(linger_us),
                                  int(admit_wait_ms), int(scratch_rows), int(mem_budget_bytes))
        h = ctypes.c_void_p()
        check(lib.ts_server_create(index.handle, ctypes.byref(p), ctypes.byref(h)))
        self._h = h
        self.index = index

    def submit(self, queries, d, t_start, t_end, max_results=0) -> int:
        lib = _lib.load()
        s, keep = make_segments(queries)
        qp = _qparams(d, t_start, t_end, max_results)
        t = ctypes.c_uint64()
        check(lib.ts_server_submit(self._h, ctypes.byref(s), ctypes.byref(qp), ctypes.byref(t)))
        del keep
        return int(t.value)

    def wait(self, ticket, timeout_ms=60000):
        """Returns (Result, timing dict); raises TsError (status 5 on timeout)."""
        lib = _lib.load()
        out = ctypes.c_void_p()
        tm = _lib.ts_request_timing()
        check(lib.ts_server_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(out),
                                 ctypes.byref(tm)))
        return Result(out, 0), {"submit_us": tm.submit_us, "start_us": tm.start_us,
                                "done_us": tm.done_us, "batch_requests": int(tm.batch_requests),
                                "requeued": int(tm.requeued)}

    def info(self) -> dict:
        """Device-memory accounting: budget, bytes held by the plans, bytes of live result rows."""
        lib = _lib.load()
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        check(lib.ts_server_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"budget_bytes": int(a.value), "plan_bytes": int(b.value),
                "held_bytes": int(c.value)}

    def cancel(self, ticket):
        check(_lib.load().ts_server_cancel(self._h, int(ticket)))

    def close(self):
        if self._h:
            _lib.load().ts_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
