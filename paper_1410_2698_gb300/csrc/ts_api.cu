// ts_api.cu -- the extern "C" boundary declared in include/ts.h.
#include <string.h>

#include <new>
#include <vector>

#include "ts_batch.cuh"
#include "ts_server.cuh"


using namespace ts;

struct ts_index {
    Index ix;
};

struct ts_result {
    uint32_t magic = MAGIC_RESULT;
    cudaStream_t stream = nullptr;
    SearchOut out;
    std::shared_ptr<RowBlock> block;  // rows shared with the other results of one batch
};

struct ts_batch {
    BatchPlan plan;
};

namespace {

ts_status clear_error(ts_status s)
{
    if (s == TS_OK) set_error("%s", "");
    return s;
}

template <class F>
ts_status guarded(F &&f)
{
    try {
        return f();
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return TS_ERR_OOM;
    } catch (...) {
        set_error("unexpected exception");
        return TS_ERR_INTERNAL;
    }
}

void free_result_arrays(ts_result *r)
{
    if (r->block) {  // rows owned by the batch's shared block
        r->block.reset();
        r->out.q = r->out.e = nullptr;
        r->out.tin = r->out.tout = nullptr;
        return;
    }
    cudaStream_t s = r->stream;
    if (r->out.q) cudaFreeAsync(r->out.q, s);
    if (r->out.e) cudaFreeAsync(r->out.e, s);
    if (r->out.tin) cudaFreeAsync(r->out.tin, s);
    if (r->out.tout) cudaFreeAsync(r->out.tout, s);
    r->out.q = r->out.e = nullptr;
    r->out.tin = r->out.tout = nullptr;
}

}  // namespace

extern "C" {

const char *ts_version(void) { return "ts_gb300 0.1 (sm_103a)"; }

const char *ts_last_error(void) { return ts::last_error(); }

ts_status ts_measure_alu_peaks(double *fp32_tflops, double *fp64_tflops)
{
    if (!fp32_tflops || !fp64_tflops) {
        set_error("ts_measure_alu_peaks: NULL argument");
        return TS_ERR_INVALID_ARG;
    }
    return guarded([&]() -> ts_status {
        ts_status st = measure_alu_peaks(fp32_tflops, fp64_tflops);
        return st == TS_OK ? clear_error(st) : st;
    });
}

ts_status ts_eval_refined_estimates(const double *x, uint64_t n, double *rcp_est,
                                     double *sqrt_est, double *rcp_ref, double *sqrt_ref)
{
    if (n && (!x || !rcp_est || !sqrt_est || !rcp_ref || !sqrt_ref)) {
        set_error("ts_eval_refined_estimates: NULL argument");
        return TS_ERR_INVALID_ARG;
    }
    return guarded([&]() -> ts_status {
        ts_status st = eval_estimates(x, n, rcp_est, sqrt_est, rcp_ref, sqrt_ref);
        return st == TS_OK ? clear_error(st) : st;
    });
}

ts_status ts_debug_inject_stall(uint64_t limit_ns)
{
    if (limit_ns == 0 || limit_ns > 1000000000ull) {
        set_error("ts_debug_inject_stall: limit must be in (0, 1e9] ns");
        return TS_ERR_INVALID_ARG;
    }
    inject_stall(limit_ns);
    return clear_error(TS_OK);
}

uint64_t ts_kernel_launches(void) { return (uint64_t)ts::launch_count(); }

ts_status ts_search_brute_noalloc(const ts_segments *db, const ts_segments *q,
                                  const ts_query_params *qp, uint32_t *q_idx, uint32_t *e_idx,
                                  double *t_in, double *t_out, uint64_t capacity, uint64_t *count,
                                  void *stream)
{
    ts_status st = ts::search_brute_noalloc(db, q, qp, q_idx, e_idx, t_in, t_out, capacity,
                                            count, (cudaStream_t)stream);
    return st == TS_OK ? clear_error(st) : st;
}

ts_status ts_build_index(const ts_segments *db, const ts_index_params *params, void *stream,
                         ts_index **out)
{
    return guarded([&]() -> ts_status {
        if (!out) {
            set_error("ts_build_index: NULL out");
            return TS_ERR_INVALID_ARG;
        }
        *out = nullptr;
        Index *ix = nullptr;
        ts_status st = build_index(db, params, (cudaStream_t)stream, &ix);
        if (st != TS_OK) return st;
        // Index is the first (only) member of ts_index: the handle is the Index object itself.
        static_assert(sizeof(ts_index) == sizeof(Index), "handle layout");
        *out = reinterpret_cast<ts_index *>(ix);
        return clear_error(TS_OK);
    });
}

ts_status ts_index_get_info(const ts_index *h, ts_index_info *info)
{
    const Index *ix = reinterpret_cast<const Index *>(h);
    if (!ix || ix->magic != MAGIC_INDEX || !info) {
        set_error("ts_index_get_info: invalid handle or NULL info");
        return TS_ERR_INVALID_ARG;
    }
    memset(info, 0, sizeof(*info));
    info->kind = ix->kind;
    info->t_bins = ix->m;
    for (int d = 0; d < 3; d++) {
        info->sub_bins[d] = ix->v[d];
        info->st_len[d] = ix->st_len[d];
        info->sub_lo[d] = ix->sub_lo[d];
        info->sub_w[d] = ix->sub_w[d];
        info->grid_lo[d] = ix->g_lo[d];
        info->grid_w[d] = ix->g_w[d];
    }
    info->grid_cells = ix->g;
    info->n = ix->n;
    info->grid_len = ix->g_len;
    info->device_bytes = ix->bytes;
    info->t_min = ix->tmin;
    info->t_max = ix->tmax;
    info->bin_width = ix->b;
    return clear_error(TS_OK);
}

ts_status ts_index_export(const ts_index *h, int32_t field, int32_t dim, void *dst,
                          uint64_t capacity, uint64_t *size)
{
    const Index *ix = reinterpret_cast<const Index *>(h);
    if (!ix || ix->magic != MAGIC_INDEX) {
        set_error("ts_index_export: invalid handle");
        return TS_ERR_INVALID_ARG;
    }
    const void *src = nullptr;
    uint64_t bytes = 0;
    bool dim_ok = dim >= 0 && dim < 3;
    switch (field) {
    case TS_FIELD_PERM: src = ix->orig; bytes = 4 * ix->n; break;
    case TS_FIELD_BIN_START: src = ix->bin_start; bytes = 8ull * ix->m; break;
    case TS_FIELD_BIN_END: src = ix->bin_end; bytes = 8ull * ix->m; break;
    case TS_FIELD_BIN_OFF: src = ix->bin_off; bytes = 4ull * (ix->m + 1ull); break;
    case TS_FIELD_ST_IDS:
        if (!dim_ok || !ix->st_ids[dim]) break;
        src = ix->st_ids[dim];
        bytes = 4 * ix->st_len[dim];
        break;
    case TS_FIELD_ST_OFF:
        if (!dim_ok || !ix->st_off[dim]) break;
        src = ix->st_off[dim];
        bytes = 4ull * ((uint64_t)ix->v[dim] * ix->m + 1ull);
        break;
    case TS_FIELD_GRID_A: src = ix->ga; bytes = 4 * ix->g_len; break;
    case TS_FIELD_GRID_OFF:
        src = ix->g_off;
        bytes = ix->g_off ? 4ull * ((uint64_t)ix->g * ix->g * ix->g + 1ull) : 0;
        break;
    default: break;
    }
    if (!src) {
        set_error("ts_index_export: field %d (dim %d) not present in this index", field, dim);
        return TS_ERR_INVALID_ARG;
    }
    if (size) *size = bytes;
    if (!dst || capacity < bytes) {
        set_error("ts_index_export: capacity %llu below %llu bytes", (unsigned long long)capacity,
                  (unsigned long long)bytes);
        return TS_ERR_CAPACITY;
    }
    TS_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
    return clear_error(TS_OK);
}

ts_status ts_schedule(const ts_index *h, const ts_segments *q, const ts_query_params *qp,
                      void *stream, int32_t *sel, uint64_t *lo, uint64_t *hi)
{
    const Index *ix = reinterpret_cast<const Index *>(h);
    if (!ix || ix->magic != MAGIC_INDEX) {
        set_error("ts_schedule: invalid index handle");
        return TS_ERR_INVALID_ARG;
    }
    return guarded([&]() -> ts_status {
        ts_status st = schedule_only(ix, q, qp, (cudaStream_t)stream, sel, lo, hi);
        return st == TS_OK ? clear_error(st) : st;
    });
}

ts_status ts_search(const ts_index *h, const ts_segments *q, const ts_query_params *qp,
                    void *stream, ts_result **out)
{
    const Index *ix = reinterpret_cast<const Index *>(h);
    if (!ix || ix->magic != MAGIC_INDEX || !out) {
        set_error("ts_search: invalid index handle or NULL out");
        return TS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    return guarded([&]() -> ts_status {
        ts_result *r = new ts_result();
        r->stream = (cudaStream_t)stream;
        ts_status st = search_plain(ix, q, qp, r->stream, &r->out);
        if (st == TS_OK || st == TS_ERR_CAPACITY) {
            *out = r;
            return st == TS_OK ? clear_error(st) : st;
        }
        free_result_arrays(r);
        delete r;
        return st;
    });
}

ts_status ts_search_points(const ts_index *h, const double *x, const double *y, const double *z,
                           uint64_t n, int32_t on_host, const ts_query_params *qp, void *stream,
                           ts_result **out)
{
    const Index *ix = reinterpret_cast<const Index *>(h);
    if (!ix || ix->magic != MAGIC_INDEX || !out) {
        set_error("ts_search_points: invalid index handle or NULL out");
        return TS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    return guarded([&]() -> ts_status {
        ts_result *r = new ts_result();
        r->stream = (cudaStream_t)stream;
        ts_status st = search_points(ix, x, y, z, n, on_host != 0, qp, r->stream, &r->out);
        if (st == TS_OK || st == TS_ERR_CAPACITY) {
            *out = r;
            return st == TS_OK ? clear_error(st) : st;
        }
        free_result_arrays(r);
        delete r;
        return st;
    });
}

ts_status ts_search_batch(const ts_index *h, uint32_t nreq, const ts_segments *qs,
                          const ts_query_params *qps, void *stream, ts_result **outs)
{
    const Index *ix = reinterpret_cast<const Index *>(h);
    if (!ix || ix->magic != MAGIC_INDEX || !outs) {
        set_error("ts_search_batch: invalid index handle or NULL outs");
        return TS_ERR_INVALID_ARG;
    }
    for (uint32_t r = 0; r < nreq; r++) outs[r] = nullptr;
    return guarded([&]() -> ts_status {
        std::vector<SearchOut> res;
        std::shared_ptr<RowBlock> block;
        ts_status st = search_batch(ix, nreq, qs, qps, (cudaStream_t)stream, res, block);
        if (st != TS_OK && st != TS_ERR_CAPACITY) return st;
        if (res.size() != nreq) {
            if (st == TS_OK) {
                set_error("ts_search_batch: internal result count mismatch");
                return TS_ERR_INTERNAL;
            }
            return st;
        }
        for (uint32_t r = 0; r < nreq; r++) {
            ts_result *o = new ts_result();
            o->stream = (cudaStream_t)stream;
            o->out = res[r];
            o->block = block;
            outs[r] = o;
        }
        return st == TS_OK ? clear_error(st) : st;
    });
}

ts_status ts_batch_create(const ts_index *h, const ts_batch_params *params, void *stream,
                          ts_batch **out)
{
    const Index *ix = reinterpret_cast<const Index *>(h);
    if (!ix || ix->magic != MAGIC_INDEX || !out) {
        set_error("ts_batch_create: invalid index handle or NULL out");
        return TS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    return guarded([&]() -> ts_status {
        BatchPlan *p = nullptr;
        ts_status st = create_plan(ix, params, (cudaStream_t)stream, true, &p);
        if (st != TS_OK) return st;
        static_assert(sizeof(ts_batch) == sizeof(BatchPlan), "handle layout");
        *out = reinterpret_cast<ts_batch *>(p);
        return clear_error(TS_OK);
    });
}

ts_status ts_batch_run(ts_batch *h, uint32_t nreq, const ts_segments *qs,
                       const ts_query_params *qps, void *stream)
{
    BatchPlan *p = reinterpret_cast<BatchPlan *>(h);
    if (!p || p->magic != MAGIC_BATCH) {
        set_error("ts_batch_run: invalid batch handle");
        return TS_ERR_INVALID_ARG;
    }
    return guarded([&]() -> ts_status {
        ts_status st = plan_run(p, nreq, qs, qps, (cudaStream_t)stream);
        return st == TS_OK ? clear_error(st) : st;
    });
}

ts_status ts_batch_wait(ts_batch *h, ts_batch_status *status)
{
    BatchPlan *p = reinterpret_cast<BatchPlan *>(h);
    if (!p || p->magic != MAGIC_BATCH) {
        set_error("ts_batch_wait: invalid batch handle");
        return TS_ERR_INVALID_ARG;
    }
    ts_status st = plan_wait(p, status);
    return st == TS_OK ? clear_error(st) : st;
}

ts_status ts_batch_request_rows(const ts_batch *h, uint32_t r, uint64_t *first, uint64_t *count)
{
    const BatchPlan *p = reinterpret_cast<const BatchPlan *>(h);
    if (!p || p->magic != MAGIC_BATCH) {
        set_error("ts_batch_request_rows: invalid batch handle");
        return TS_ERR_INVALID_ARG;
    }
    return plan_request_rows(p, r, first, count);
}

ts_status ts_batch_rows(const ts_batch *h, const uint32_t **q_idx, const uint32_t **e_idx,
                        const double **t_in, const double **t_out)
{
    const BatchPlan *p = reinterpret_cast<const BatchPlan *>(h);
    if (!p || p->magic != MAGIC_BATCH) {
        set_error("ts_batch_rows: invalid batch handle");
        return TS_ERR_INVALID_ARG;
    }
    if (q_idx) *q_idx = p->b.out_q;
    if (e_idx) *e_idx = p->b.out_e;
    if (t_in) *t_in = p->b.out_tin;
    if (t_out) *t_out = p->b.out_tout;
    return TS_OK;
}

ts_status ts_batch_copy_rows(const ts_batch *h, uint64_t first, uint64_t count, uint32_t *q_idx,
                             uint32_t *e_idx, double *t_in, double *t_out)
{
    const BatchPlan *p = reinterpret_cast<const BatchPlan *>(h);
    if (!p || p->magic != MAGIC_BATCH) {
        set_error("ts_batch_copy_rows: invalid batch handle");
        return TS_ERR_INVALID_ARG;
    }
    if (first + count > p->caps.rows || first + count < first) {
        set_error("ts_batch_copy_rows: rows beyond the plan's capacity");
        return TS_ERR_INVALID_ARG;
    }
    // on the plan's own stream, after its last run: a stream the plan shares with later work
    // (plans run one after another) keeps running while the rows are read
    cudaStream_t s = p->stream;
    if (p->done) TS_CUDA(cudaStreamWaitEvent(s, p->done, 0));
    if (count) {
        if (q_idx) TS_CUDA(cudaMemcpyAsync(q_idx, p->b.out_q + first, 4 * count, cudaMemcpyDeviceToHost, s));
        if (e_idx) TS_CUDA(cudaMemcpyAsync(e_idx, p->b.out_e + first, 4 * count, cudaMemcpyDeviceToHost, s));
        if (t_in) TS_CUDA(cudaMemcpyAsync(t_in, p->b.out_tin + first, 8 * count, cudaMemcpyDeviceToHost, s));
        if (t_out) TS_CUDA(cudaMemcpyAsync(t_out, p->b.out_tout + first, 8 * count, cudaMemcpyDeviceToHost, s));
    }
    TS_CUDA(cudaStreamSynchronize(s));
    return clear_error(TS_OK);
}

ts_status ts_server_create(const ts_index *h, const ts_server_params *params, ts_server **out)
{
    const Index *ix = reinterpret_cast<const Index *>(h);
    if (!ix || ix->magic != MAGIC_INDEX || !out) {
        set_error("ts_server_create: invalid index handle or NULL out");
        return TS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    return guarded([&]() -> ts_status {
        Server *s = nullptr;
        ts_status st = server_create(ix, params, &s);
        if (st != TS_OK) return st;
        *out = reinterpret_cast<ts_server *>(s);
        return clear_error(TS_OK);
    });
}

static Server *as_server(ts_server *h)
{
    Server *s = reinterpret_cast<Server *>(h);
    if (!s || *reinterpret_cast<uint32_t *>(s) != MAGIC_SERVER) return nullptr;
    return s;
}

ts_status ts_server_submit(ts_server *h, const ts_segments *q, const ts_query_params *qp,
                           uint64_t *ticket)
{
    Server *s = as_server(h);
    if (!s) {
        set_error("ts_server_submit: invalid server handle");
        return TS_ERR_INVALID_ARG;
    }
    return guarded([&]() -> ts_status { return server_submit(s, q, qp, ticket); });
}

ts_status ts_server_wait(ts_server *h, uint64_t ticket, uint32_t timeout_ms, ts_result **out,
                         ts_request_timing *timing)
{
    Server *s = as_server(h);
    if (!s || !out) {
        set_error("ts_server_wait: invalid server handle or NULL out");
        return TS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    return guarded([&]() -> ts_status {
        SearchOut o;
        std::shared_ptr<RowBlock> block;
        ts_status st = server_wait(s, ticket, timeout_ms, &o, &block, timing);
        if (st != TS_OK) return st;
        ts_result *r = new ts_result();
        r->stream = nullptr;
        r->out = o;
        r->block = block;
        *out = r;
        return clear_error(TS_OK);
    });
}

ts_status ts_server_info(ts_server *srv, uint64_t *budget_bytes, uint64_t *plan_bytes,
                         uint64_t *held_bytes)
{
    Server *s = as_server(srv);
    if (!s) {
        set_error("ts_server_info: invalid server handle");
        return TS_ERR_INVALID_ARG;
    }
    server_info(s, budget_bytes, plan_bytes, held_bytes);
    return clear_error(TS_OK);
}

ts_status ts_server_cancel(ts_server *h, uint64_t ticket)
{
    Server *s = as_server(h);
    if (!s) {
        set_error("ts_server_cancel: invalid server handle");
        return TS_ERR_INVALID_ARG;
    }
    return server_cancel(s, ticket);
}

void ts_server_destroy(ts_server *h)
{
    Server *s = as_server(h);
    if (s) server_destroy(s);
}

uint64_t ts_result_count(const ts_result *r)
{
    if (!r || r->magic != MAGIC_RESULT) return 0;
    return r->out.count;
}

ts_status ts_result_arrays(const ts_result *r, const uint32_t **q_idx, const uint32_t **e_idx,
                           const double **t_in, const double **t_out)
{
    if (!r || r->magic != MAGIC_RESULT) {
        set_error("ts_result_arrays: invalid handle");
        return TS_ERR_INVALID_ARG;
    }
    if (q_idx) *q_idx = r->out.q;
    if (e_idx) *e_idx = r->out.e;
    if (t_in) *t_in = r->out.tin;
    if (t_out) *t_out = r->out.tout;
    return clear_error(TS_OK);
}

ts_status ts_result_stats(const ts_result *r, ts_search_stats *stats)
{
    if (!r || r->magic != MAGIC_RESULT || !stats) {
        set_error("ts_result_stats: invalid handle or NULL stats");
        return TS_ERR_INVALID_ARG;
    }
    *stats = r->out.stats;
    return clear_error(TS_OK);
}

ts_status ts_result_copy_to_host(const ts_result *r, uint32_t *q_idx, uint32_t *e_idx,
                                 double *t_in, double *t_out, void *stream)
{
    if (!r || r->magic != MAGIC_RESULT) {
        set_error("ts_result_copy_to_host: invalid handle");
        return TS_ERR_INVALID_ARG;
    }
    const uint64_t n = r->out.count;
    cudaStream_t s = (cudaStream_t)stream;
    if (n && r->out.q) {
        if (q_idx) TS_CUDA(cudaMemcpyAsync(q_idx, r->out.q, 4 * n, cudaMemcpyDeviceToHost, s));
        if (e_idx) TS_CUDA(cudaMemcpyAsync(e_idx, r->out.e, 4 * n, cudaMemcpyDeviceToHost, s));
        if (t_in) TS_CUDA(cudaMemcpyAsync(t_in, r->out.tin, 8 * n, cudaMemcpyDeviceToHost, s));
        if (t_out) TS_CUDA(cudaMemcpyAsync(t_out, r->out.tout, 8 * n, cudaMemcpyDeviceToHost, s));
    }
    TS_CUDA(cudaStreamSynchronize(s));
    return clear_error(TS_OK);
}

void ts_free(void *handle)
{
    if (!handle) return;
    uint32_t magic = *reinterpret_cast<uint32_t *>(handle);
    if (magic == MAGIC_INDEX) {
        destroy_index(reinterpret_cast<Index *>(handle));
    } else if (magic == MAGIC_BATCH) {
        destroy_plan(reinterpret_cast<BatchPlan *>(handle));
    } else if (magic == MAGIC_RESULT) {
        ts_result *r = reinterpret_cast<ts_result *>(handle);
        free_result_arrays(r);
        r->magic = 0;
        delete r;
    }
}

}  // extern "C"
