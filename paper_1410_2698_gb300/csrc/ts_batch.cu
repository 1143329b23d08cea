// ts_batch.cu -- batched search: one pipeline for many requests, and reusable plans whose runs are
// captured once in a CUDA graph and replayed.
//
// A plan owns device memory for fixed capacities (queries, candidate ranges, groups, tiles, rows)
// and mapped pinned host memory for the per-run request table and the run's outcome. A run:
//   request table + run header (H2D, fixed size) -> gather the requests' query columns into the
//   plan's columns (device pointers or mapped pinned staging) -> query preparation -> sort of the
//   candidate ranges -> groups and tiles -> pair kernel count pass -> scan -> pair kernel write
//   pass -> per-request row offsets -> outcome (D2H into mapped pinned memory).
// Every size is read from the run header on the device, so the same graph serves any batch within
// the capacities; a capacity that is exceeded is reported in the outcome and no rows are written.
#include <string.h>

#include <memory>
#include <vector>

#include "ts_batch.cuh"

namespace ts {

namespace {

constexpr int TPB = 256;

static_assert(sizeof(ReqDesc) % 4 == 0, "the request table is copied as 32-bit words");

// Start of a run: the request table and the run header come from the plan's mapped pinned
// memory (written by the host before the launch), and the run's counters are reset.
__global__ void k_run_start(const ReqDesc *h_reqs, const uint32_t *h_run, ReqDesc *d_reqs,
                            uint32_t *d_run, uint32_t nreq_cap, PipeBufs b)
{
    pdl_enter();
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t words = (uint64_t)nreq_cap * (sizeof(ReqDesc) / 4);
    const uint32_t *src = reinterpret_cast<const uint32_t *>(h_reqs);
    uint32_t *dst = reinterpret_cast<uint32_t *>(d_reqs);
    for (uint64_t i = tid; i < words; i += nth) dst[i] = src[i];
    for (uint64_t i = tid; i < nreq_cap; i += nth) b.req_units[i] = 0;
    if (tid < 4) d_run[tid] = h_run[tid];
    if (tid < ST_NSLOTS) b.stats[tid] = 0;
    if (tid == 0) {
        b.status[0] = 0;
        b.counters[0] = 0;
        b.counters[1] = 0;
    }
}

// Row range of every request: its rows start at the offset of its first tile (groups of a
// request are contiguous, and so are their tiles and rows).
// (also the run's outcome -- header, statistics, status -- into the plan's mapped pinned memory,
// where the host reads it after the stream synchronised)
__global__ void k_req_rows(const uint32_t *run, uint32_t nreq_cap, uint64_t tcap, PipeBufs b,
                           unsigned long long *row0, BatchOut *out)
{
    pdl_enter();
    const uint32_t nreq = min(run[1], nreq_cap);
    const uint64_t T = (uint64_t)b.hdr[HDR_T_LO] | ((uint64_t)b.hdr[HDR_T_HI] << 32);
    const bool ok = T <= tcap;
    for (uint32_t r = threadIdx.x; r <= nreq; r += blockDim.x) {
        const uint64_t t0 = b.tile_base[b.gstart[r]];
        row0[r] = ok ? b.tile_off[t0 < T ? t0 : T] : 0ull;
    }
    if (threadIdx.x < 8) out->hdr[threadIdx.x] = b.hdr[threadIdx.x];
    if (threadIdx.x < ST_NSLOTS) out->stats[threadIdx.x] = b.stats[threadIdx.x];
    if (threadIdx.x == 0) out->status = b.status[0];
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carves one device allocation into the plan's buffers.
struct Carver {
    size_t off = 0;
    unsigned char *base = nullptr;
    template <class T>
    T *take(uint64_t count)
    {
        size_t at = off;
        off += align256(sizeof(T) * (count ? count : 1));
        return base ? reinterpret_cast<T *>(base + at) : nullptr;
    }
};

}  // namespace

// Layout of the device memory and pointers of a plan (the same code sizes and carves).
static void layout(BatchPlan *p, Carver &c)
{
    const PipeCaps &k = p->caps;
    const bool grid = p->ix->kind == TS_INDEX_SPATIAL;
    PipeBufs &b = p->b;
    b.qd = c.take<QueryD>(k.nq);
    b.qf = c.take<float4>(2 * k.nq);
    b.qreq = c.take<uint32_t>(k.nq);
    b.qcell = grid ? c.take<uint32_t>(2 * k.nq) : nullptr;
    b.qnu = grid ? c.take<uint32_t>(k.nq) : nullptr;
    b.quoff = grid ? c.take<uint32_t>(k.nq + 1) : nullptr;
    b.u_q = c.take<uint32_t>(k.units);
    b.u_lo = c.take<uint32_t>(k.units);
    b.u_hi = c.take<uint32_t>(k.units);
    b.u_sel = c.take<uint32_t>(k.units);
    b.keys = c.take<uint64_t>(k.units);
    b.vals = c.take<uint32_t>(k.units);
    b.req_units = c.take<uint32_t>(k.nreq);
    b.ustart = c.take<uint32_t>(k.nreq + 1);
    b.req_groups = c.take<uint32_t>(k.nreq);
    b.gstart = c.take<uint32_t>(k.nreq + 1);
    b.g_first = c.take<uint32_t>(k.groups);
    b.g_count = c.take<uint32_t>(k.groups);
    b.g_nseg = c.take<uint32_t>(k.groups);
    b.gmem = c.take<MemberRec>(GROUP * k.groups);
    b.ghdr = c.take<float4>(k.groups);
    b.seg_lo = c.take<uint32_t>(GROUP * k.groups);
    b.seg_hi = c.take<uint32_t>(GROUP * k.groups);
    b.seg_sel = c.take<uint32_t>(GROUP * k.groups);
    b.seg_t0 = c.take<uint32_t>(GROUP * k.groups);
    b.ntiles = c.take<uint32_t>(k.groups);
    b.tile_base = c.take<uint64_t>(k.groups + 1);
    b.tdesc = c.take<uint4>(k.tiles);
    b.s_tile = c.take<uint32_t>(k.scratch);
    b.s_rank = c.take<uint32_t>(k.scratch);
    b.s_q = c.take<uint32_t>(k.scratch);
    b.s_e = c.take<uint32_t>(k.scratch);
    b.s_tin = c.take<double>(k.scratch);
    b.s_tout = c.take<double>(k.scratch);
    b.tile_hits = c.take<uint32_t>(k.tiles);
    b.tile_off = c.take<uint64_t>(k.tiles + 1);
    if (p->own_rows) {
        b.out_q = c.take<uint32_t>(k.rows);
        b.out_e = c.take<uint32_t>(k.rows);
        b.out_tin = c.take<double>(k.rows);
        b.out_tout = c.take<double>(k.rows);
    }
    b.hdr = c.take<uint32_t>(8);
    b.stats = c.take<unsigned long long>(ST_NSLOTS);
    b.status = c.take<uint32_t>(4);
    b.counters = b.status + 1;
    p->d_reqs = c.take<ReqDesc>(k.nreq);
    p->d_run = c.take<uint32_t>(4);
    b.run = p->d_run;
}

void destroy_plan(BatchPlan *p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->dmem) cudaFree(p->dmem);
    if (p->hmem) cudaFreeHost(p->hmem);
    if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
    for (int e = 0; e < 4; e++)
        if (p->ev[e]) cudaEventDestroy(p->ev[e]);
    if (p->done) cudaEventDestroy(p->done);
    p->magic = 0;
    delete p;
}

ts_status create_plan(const Index *ix, const ts_batch_params *prm, cudaStream_t s, bool own_rows,
                      BatchPlan **out)
{
    *out = nullptr;
    if (!prm || prm->max_requests == 0 || prm->max_queries == 0 ||
        prm->max_requests >= (1u << 24) || prm->max_queries > 0x7fffffffull ||
        (own_rows && prm->max_rows == 0)) {
        set_error("batch plan: need max_requests (< 2^24), max_queries (< 2^31) and max_rows > 0");
        return TS_ERR_INVALID_ARG;
    }
    const uint32_t tile = prm->tile_records ? prm->tile_records : (uint32_t)PK_TILE;
    if (tile % PK_CH != 0 || tile > 32 * PK_CH) {
        set_error("batch plan: tile_records must be a multiple of %d, at most %d", PK_CH,
                  32 * PK_CH);
        return TS_ERR_INVALID_ARG;
    }
    std::unique_ptr<BatchPlan, void (*)(BatchPlan *)> p(new BatchPlan(), destroy_plan);
    p->ix = ix;
    p->prm = *prm;
    p->own_rows = own_rows;
    PipeCaps &k = p->caps;
    k.nq = prm->max_queries;
    k.nreq = prm->max_requests;
    k.tile = tile;
    k.pair_blocks = prm->pair_blocks;
    const bool grid = ix->kind == TS_INDEX_SPATIAL;
    k.units = prm->max_units ? prm->max_units : (grid ? 16 * k.nq : k.nq);
    k.groups = k.units / GROUP + k.nreq + 1;
    k.tiles = prm->max_tiles ? prm->max_tiles : 256 * k.groups + 65536;  // 28 B per tile
    k.rows = own_rows ? prm->max_rows : ~0ull;
    // hits the count pass keeps for placement after the scan; more hits than this make the
    // write pass sweep the tiles again
    k.scratch = prm->scratch_rows ? prm->scratch_rows
                : own_rows       ? prm->max_rows
                                 : std::min<uint64_t>(4 * k.nq + (1ull << 20), SCRATCH_MAX);
    Carver sz;
    layout(p.get(), sz);
    p->dbytes = sz.off;
    TS_CUDA(cudaMalloc(&p->dmem, p->dbytes));
    Carver cv;
    cv.base = static_cast<unsigned char *>(p->dmem);
    layout(p.get(), cv);
    // pinned, device-mapped host memory: request table, run header, query staging, outcome
    const size_t h_reqs = align256(sizeof(ReqDesc) * k.nreq);
    const size_t h_run = 256;
    const size_t h_stage = align256(sizeof(double) * 8 * k.nq);
    const size_t h_out = align256(sizeof(BatchOut)) + align256(8 * (k.nreq + 1));
    p->hbytes = h_reqs + h_run + h_stage + h_out;
    TS_CUDA(cudaHostAlloc(&p->hmem, p->hbytes, cudaHostAllocMapped | cudaHostAllocPortable));
    unsigned char *h = static_cast<unsigned char *>(p->hmem);
    p->h_reqs = reinterpret_cast<ReqDesc *>(h);
    p->h_run = reinterpret_cast<uint32_t *>(h + h_reqs);
    p->h_stage = reinterpret_cast<double *>(h + h_reqs + h_run);
    p->h_out = reinterpret_cast<BatchOut *>(h + h_reqs + h_run + h_stage);
    p->h_row0 = reinterpret_cast<unsigned long long *>(h + h_reqs + h_run + h_stage +
                                                       align256(sizeof(BatchOut)));
    memset(p->hmem, 0, p->hbytes);
    // device views of the mapped pinned memory (the run's first and last kernels use them)
    {
        void *dh = nullptr;
        TS_CUDA(cudaHostGetDevicePointer(&dh, p->hmem, 0));
        unsigned char *d = static_cast<unsigned char *>(dh);
        unsigned char *hb = static_cast<unsigned char *>(p->hmem);
        p->dh_reqs = reinterpret_cast<ReqDesc *>(d + (reinterpret_cast<unsigned char *>(p->h_reqs) - hb));
        p->dh_run = reinterpret_cast<uint32_t *>(d + (reinterpret_cast<unsigned char *>(p->h_run) - hb));
        p->dh_out = reinterpret_cast<BatchOut *>(d + (reinterpret_cast<unsigned char *>(p->h_out) - hb));
        p->dh_row0 = reinterpret_cast<unsigned long long *>(
            d + (reinterpret_cast<unsigned char *>(p->h_row0) - hb));
        p->dh_stage =
            reinterpret_cast<double *>(d + (reinterpret_cast<unsigned char *>(p->h_stage) - hb));
    }
    if (s) {
        p->stream = s;
    } else {
        TS_CUDA(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
        p->own_stream = true;
    }
    TS_CUDA(cudaMemsetAsync(p->dmem, 0, p->dbytes, p->stream));
    TS_CUDA(cudaStreamSynchronize(p->stream));
    for (int e = 0; e < 4; e++) TS_CUDA(cudaEventCreate(&p->ev[e]));
    TS_CUDA(cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming));
    *out = p.release();
    return TS_OK;
}

// Stage a run's request table and query columns (host side). Returns the query count.
static ts_status stage_requests(BatchPlan *p, uint32_t nreq, const ts_segments *qs,
                                const ts_query_params *qps, uint64_t *nq_out)
{
    const PipeCaps &k = p->caps;
    if (nreq == 0 || nreq > k.nreq || !qs || !qps) {
        set_error("batch run: nreq must be in [1, %u]", k.nreq);
        return TS_ERR_INVALID_ARG;
    }
    uint64_t nq = 0;
    for (uint32_t r = 0; r < nreq; r++) {
        TS_CHECK(check_query_params(&qps[r]));
        nq += qs[r].n;
    }
    if (nq > k.nq) {
        set_error("batch run: %llu query segments exceed the plan's %llu",
                  (unsigned long long)nq, (unsigned long long)k.nq);
        return TS_ERR_CAPACITY;
    }
    uint64_t first = 0;
    for (uint32_t r = 0; r < nreq; r++) {
        ReqDesc &R = p->h_reqs[r];
        fill_req(R, &qps[r], (uint32_t)first, (uint32_t)qs[r].n);
        const double *src[8] = {qs[r].x0, qs[r].y0, qs[r].z0, qs[r].t0,
                                qs[r].x1, qs[r].y1, qs[r].z1, qs[r].t1};
        for (int c = 0; c < 8; c++) {
            if (!src[c] && qs[r].n) {
                set_error("batch run: NULL column %d of request %u", c, r);
                return TS_ERR_INVALID_ARG;
            }
            if (qs[r].on_host) {
                // pinned (page-locked, mapped) host columns are read by the device in place;
                // other host memory is copied into the plan's mapped staging area
                cudaPointerAttributes pa;
                void *dev = nullptr;
                if (qs[r].n && cudaPointerGetAttributes(&pa, src[c]) == cudaSuccess &&
                    pa.type == cudaMemoryTypeHost &&
                    cudaHostGetDevicePointer(&dev, const_cast<double *>(src[c]), 0) ==
                        cudaSuccess) {
                    R.cols[c] = static_cast<const double *>(dev);
                    continue;
                }
                cudaGetLastError();  // (pageable memory: not an error)
                double *dst = p->h_stage + (uint64_t)c * k.nq + first;
                if (qs[r].n) memcpy(dst, src[c], sizeof(double) * qs[r].n);
                R.cols[c] = p->dh_stage + (uint64_t)c * k.nq + first;
            } else {
                R.cols[c] = src[c];
            }
        }
        first += qs[r].n;
    }
    // unused request slots: empty, after every query
    for (uint32_t r = nreq; r < k.nreq; r++) {
        ts_query_params z{1.0, 0.0, 0.0, 0};
        fill_req(p->h_reqs[r], &z, (uint32_t)nq, 0);
        for (int c = 0; c < 8; c++) p->h_reqs[r].cols[c] = nullptr;
    }
    p->h_run[0] = (uint32_t)nq;
    p->h_run[1] = nreq;
    *nq_out = nq;
    return TS_OK;
}

// Enqueue the run (no host synchronisation; graph-capturable). With write = false the run stops
// after the scan (one-shot batches size their rows first).
// Records a timing event; inside a stream capture the event becomes an event-record node of the
// graph (cudaEventRecordExternal), so that replays time the passes too.
static cudaError_t record_ev(cudaEvent_t e, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cs);
    if (ce != cudaSuccess) return ce;
    return cs == cudaStreamCaptureStatusActive
               ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
               : cudaEventRecord(e, s);
}

static ts_status enqueue_run(BatchPlan *p, cudaStream_t s, bool write)
{
    const PipeCaps &k = p->caps;
    const PipeBufs &b = p->b;
    const bool grid = p->ix->kind == TS_INDEX_SPATIAL;
    {
        const uint64_t words = (uint64_t)k.nreq * (sizeof(ReqDesc) / 4);
        const unsigned sb = (unsigned)std::min<uint64_t>((words + TPB - 1) / TPB + 1, 64);
        TS_LAUNCH_PDL(k_run_start, dim3(sb), dim3(TPB), 0, s,
                      p->dh_reqs, p->dh_run, p->d_reqs, p->d_run, k.nreq, b);
    }
    // every stage below sizes its work from the run's counts in device memory (the header and
    // the run header), not from the plan's capacities; the queries are read through the
    // request table
    TS_CHECK(pipe_prepare(p->ix, nullptr, k.nq, p->d_reqs, k.nreq, b, k, s));
    if (grid) {
        TS_CHECK(scan_u32(b.qnu, b.quoff, k.nq, b.status, s, p->d_run));
        TS_CHECK(pipe_grid_units(p->ix, k.nq, b, k, s));
    }
    TS_CHECK(pipe_group(p->ix, p->d_reqs, k.nreq, b, k, false, s));
    TS_CUDA(record_ev(p->ev[0], s));
    TS_CHECK(pipe_count(p->ix, p->d_reqs, b, k, s));
    TS_CUDA(record_ev(p->ev[1], s));
    TS_CHECK(pipe_scan_rows(b, k, s));
    if (write) {
        TS_CUDA(record_ev(p->ev[2], s));
        TS_CHECK(pipe_write(p->ix, p->d_reqs, b, k, s));
        TS_CUDA(record_ev(p->ev[3], s));
    }
    TS_LAUNCH_PDL(k_req_rows, dim3(1), dim3(256), 0, s,
                  p->d_run, k.nreq, k.tiles, b, p->dh_row0, p->dh_out);
    return TS_OK;
}

ts_status plan_run(BatchPlan *p, uint32_t nreq, const ts_segments *qs, const ts_query_params *qps,
                   cudaStream_t s)
{
    if (p->running) {
        set_error("batch run: the previous run has not been waited for");
        return TS_ERR_INVALID_ARG;
    }
    uint64_t nq = 0;
    TS_CHECK(stage_requests(p, nreq, qs, qps, &nq));
    cudaStream_t st = s ? s : p->stream;
    if (p->prm.use_graph) {
        if (!p->exec) {
            // kernels enqueued during the capture are counted once, for this first replay
            const unsigned long long before = launch_count();
            TS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            ts_status e = enqueue_run(p, st, p->own_rows);
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamEndCapture(st, &g);
            if (e != TS_OK) {
                if (g) cudaGraphDestroy(g);
                return e;
            }
            if (ce != cudaSuccess) return cuda_status(ce, "cudaStreamEndCapture");
            p->graph = g;
            p->graph_kernels = launch_count() - before;
            TS_CUDA(cudaGraphInstantiate(&p->exec, g, 0));
        } else {
            note_launches(p->graph_kernels);
        }
        TS_CUDA(cudaGraphLaunch(p->exec, st));
    } else {
        TS_CHECK(enqueue_run(p, st, p->own_rows));
    }
    TS_CUDA(cudaEventRecord(p->done, st));
    p->running = true;
    p->last_nreq = nreq;
    return TS_OK;
}

static void fill_stats(const BatchOut *o, ts_search_stats *s)
{
    memset(s, 0, sizeof(*s));
    s->n_qsegs = o->stats[ST_QSEGS];
    s->n_tests = o->stats[ST_TESTS];
    s->n_exact = o->stats[ST_EXACT];
    s->n_hits = o->stats[ST_HITS];
    s->n_tiles = o->stats[ST_TILES];
    s->n_groups = o->stats[ST_GROUPS];
    s->n_subbin = o->stats[ST_SUBBIN];
    s->n_chunks = o->stats[ST_CHUNKS];
    s->n_dense = o->stats[ST_DENSE];
    s->n_sparse = o->stats[ST_SPARSE];
    s->n_stage2 = o->stats[ST_STAGE2];
}

ts_status plan_wait(BatchPlan *p, ts_batch_status *out)
{
    if (!p->running) {
        set_error("batch wait: no run in flight");
        return TS_ERR_INVALID_ARG;
    }
    TS_CUDA(cudaEventSynchronize(p->done));
    p->running = false;
    const uint32_t st = p->h_out->status;
    ts_batch_status bs;
    memset(&bs, 0, sizeof(bs));
    bs.nreq = p->last_nreq;
    bs.rows = p->h_out->stats[ST_HITS];
    bs.overflow = (st & DEV_ERR_OVERFLOW) ? 1 : 0;
    fill_stats(p->h_out, &bs.stats);
    bs.stats.n_queries = p->h_run[0];
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev[0], p->ev[1]) == cudaSuccess) bs.stats.ms_count_pass = ms;
    if (cudaEventElapsedTime(&ms, p->ev[2], p->ev[3]) == cudaSuccess) bs.stats.ms_write_pass = ms;
    cudaGetLastError();  // a run without a write pass leaves ev[2..3] unrecorded
    if (out) *out = bs;
    if (st & ~DEV_ERR_OVERFLOW) return read_dev_status(st & ~DEV_ERR_OVERFLOW);
    return TS_OK;
}

ts_status plan_request_rows(const BatchPlan *p, uint32_t r, uint64_t *first, uint64_t *count)
{
    if (r >= p->last_nreq) {
        set_error("batch rows: request %u of %u", r, p->last_nreq);
        return TS_ERR_INVALID_ARG;
    }
    const unsigned long long a = p->h_row0[r], b = p->h_row0[r + 1];
    if (first) *first = a;
    if (count) *count = b - a;
    return TS_OK;
}

// One-shot batch with exact-size rows shared by the per-request results.
ts_status search_batch(const Index *ix, uint32_t nreq, const ts_segments *qs,
                       const ts_query_params *qps, cudaStream_t s,
                       std::vector<SearchOut> &outs, std::shared_ptr<RowBlock> &block)
{
    if (nreq == 0 || !qs || !qps) {
        set_error("ts_search_batch: need nreq > 0 and arrays of requests");
        return TS_ERR_INVALID_ARG;
    }
    uint64_t nq = 0;
    for (uint32_t r = 0; r < nreq; r++) nq += qs[r].n;
    ts_batch_params prm;
    memset(&prm, 0, sizeof(prm));
    prm.max_requests = nreq;
    prm.max_queries = nq ? nq : 1;
    std::unique_ptr<BatchPlan, void (*)(BatchPlan *)> p(nullptr, destroy_plan);
    cudaStream_t st = nullptr;
    uint32_t status = 0;
    // exact sizing: when the candidate ranges or tiles outgrow the first guess, the plan is
    // rebuilt with the sizes the device reported
    for (int attempt = 0; attempt < 3; attempt++) {
        BatchPlan *raw = nullptr;
        TS_CHECK(create_plan(ix, &prm, s, false, &raw));
        p.reset(raw);
        uint64_t staged = 0;
        TS_CHECK(stage_requests(p.get(), nreq, qs, qps, &staged));
        st = p->stream;
        TS_CHECK(enqueue_run(p.get(), st, false));
        TS_CUDA(cudaStreamSynchronize(st));
        status = p->h_out->status;
        if (!(status & DEV_ERR_OVERFLOW)) break;
        const uint64_t tiles = (uint64_t)p->h_out->hdr[HDR_T_LO] |
                               ((uint64_t)p->h_out->hdr[HDR_T_HI] << 32);
        if (p->b.quoff) {
            uint32_t units = 0;
            TS_CUDA(cudaMemcpy(&units, p->b.quoff + p->caps.nq, 4, cudaMemcpyDeviceToHost));
            prm.max_units = std::max<uint64_t>(units, p->caps.units);
        }
        prm.max_tiles = std::max<uint64_t>(2 * tiles, p->caps.tiles);
    }
    if (status) return read_dev_status(status);
    const uint64_t total = p->h_out->stats[ST_HITS];
    outs.assign(nreq, SearchOut{});
    bool over = false;
    for (uint32_t r = 0; r < nreq; r++) {
        outs[r].count = p->h_row0[r + 1] - p->h_row0[r];
        outs[r].stats.n_queries = qs[r].n;
        outs[r].stats.n_hits = outs[r].count;
        if (qps[r].max_results && outs[r].count > qps[r].max_results) over = true;
    }
    if (over) {
        set_error("ts_search_batch: a request's rows exceed its max_results");
        return TS_ERR_CAPACITY;
    }
    if (total) {
        block = std::make_shared<RowBlock>();
        TS_CHECK(block->alloc(total, st));
        p->b.out_q = block->q;
        p->b.out_e = block->e;
        p->b.out_tin = block->tin;
        p->b.out_tout = block->tout;
        p->caps.rows = total;
        TS_CHECK(pipe_write(ix, p->d_reqs, p->b, p->caps, st));
        TS_CUDA(cudaMemcpyAsync(&p->h_out->status, p->b.status, 4, cudaMemcpyDeviceToHost, st));
        TS_CUDA(cudaStreamSynchronize(st));
        status = p->h_out->status;
        if (status) return read_dev_status(status);
        for (uint32_t r = 0; r < nreq; r++) {
            const uint64_t a = p->h_row0[r];
            outs[r].q = block->q + a;
            outs[r].e = block->e + a;
            outs[r].tin = block->tin + a;
            outs[r].tout = block->tout + a;
        }
    }
    return TS_OK;
}

ts_status RowBlock::alloc(uint64_t n, cudaStream_t s)
{
    TS_CUDA(pool_malloc((void **)&q, sizeof(uint32_t) * n, s));
    TS_CUDA(pool_malloc((void **)&e, sizeof(uint32_t) * n, s));
    TS_CUDA(pool_malloc((void **)&tin, sizeof(double) * n, s));
    TS_CUDA(pool_malloc((void **)&tout, sizeof(double) * n, s));
    bytes = ROW_BYTES * n;
    if (held) held->fetch_add((int64_t)bytes);
    return TS_OK;
}

// The rows are handed out only after the kernels that wrote them completed; the memory goes
// back to the library's pool.
RowBlock::~RowBlock()
{
    if (q) cudaFreeAsync(q, 0);
    if (e) cudaFreeAsync(e, 0);
    if (tin) cudaFreeAsync(tin, 0);
    if (tout) cudaFreeAsync(tout, 0);
    if (held && bytes) held->fetch_sub((int64_t)bytes);
}

}  // namespace ts
