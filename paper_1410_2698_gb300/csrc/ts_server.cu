// ts_server.cu -- the served search: a request loop on a resident index with continuous batching.
//
// Client threads submit requests (their query segments are copied into the request); one loop
// thread forms batches from the queue in arrival order while a batch's request and query
// capacities allow, and runs them on up to max_inflight batch plans, each with its own stream:
// requests that arrive while a batch is on the device go into the next free plan, so batches
// overlap on the device. A batch runs in two phases: its plan (a CUDA graph) runs up to the count
// pass and the row scan; the loop then admits the batch's exact rows against the server's
// device-memory budget (its plans plus the rows of results not yet released) -- a batch whose
// rows do not fit beside the rows still held waits, its plan idle, until results are released --
// allocates them from the library's pool and launches the write phase into them. A batch with
// more rows than max_batch_rows or than the budget holds, or that outgrew a work capacity, is
// split or its plan grown, and re-run; a lone request that cannot fit ends with TS_ERR_CAPACITY.
// Completed requests share the batch's row block (each result is a view of its rows) and carry
// host timestamps. Every wait -- client waits and the loop's idle waits -- is bounded.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ts_batch.cuh"
#include "ts_server.cuh"

namespace ts {

namespace {

enum { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2 };

struct SrvReq {
    uint64_t ticket = 0;
    std::vector<double> cols;  // 8 columns of n values
    uint64_t n = 0;
    ts_query_params qp{};
    double submit_us = 0, start_us = 0, done_us = 0;
    uint32_t batch_requests = 0;
    uint32_t requeued = 0;  // times its batch went back to the queue
    int state = RQ_QUEUED;
    ts_status status = TS_OK;
    std::string error;
    SearchOut out;
    std::shared_ptr<RowBlock> block;  // the batch's rows (out points into them)
};

// A slot's phases: its batch's count phase on the device, waiting for room in the memory
// budget for its rows (the plan idle, holding the count phase's offsets), the write phase.
enum { SLOT_IDLE = 0, SLOT_COUNT = 1, SLOT_ADMIT = 2, SLOT_WRITE = 3 };

struct Slot {
    BatchPlan *plan = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<SrvReq *> batch;
    bool busy = false;
    int phase = SLOT_IDLE;
    uint64_t rows = 0;  // the batch's rows (count phase done)
    double admit_since_us = 0;  // when the batch started waiting for room in the budget
    std::shared_ptr<RowBlock> block;
};

}  // namespace

struct Server {
    uint32_t magic = MAGIC_SERVER;
    const Index *ix = nullptr;
    ts_server_params prm{};
    int device = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<SrvReq *> queue;
    std::unordered_map<uint64_t, SrvReq *> reqs;
    std::thread th;
    std::atomic<bool> stop{false};  // set under mu; read also by the loop outside it
    uint64_t next_ticket = 1;
    size_t split_limit = 0;  // after an overflow: at most this many requests in the next batch
    // device-memory budget: the plans' own bytes, and the bytes of live row blocks (updated by
    // the blocks themselves, also after the server is gone)
    uint64_t budget = 0, plan_bytes = 0;
    std::shared_ptr<std::atomic<int64_t>> held = std::make_shared<std::atomic<int64_t>>(0);
    std::chrono::steady_clock::time_point t0;

    uint64_t row_budget() const { return budget > plan_bytes ? budget - plan_bytes : 0; }

    double now_us() const
    {
        return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0)
            .count();
    }
};

namespace {

void end_request(Server *s, SrvReq *r, ts_status st, const char *msg)
{
    r->status = st;
    if (msg) r->error = msg;
    r->state = RQ_DONE;
    r->done_us = s->now_us();
}

// Re-queue a batch at the front, in order; the next batches take half as many requests. A lone
// request that cannot fit ends with TS_ERR_CAPACITY. (Caller holds the lock.)
void split_batch(Server *s, std::vector<SrvReq *> &batch, const char *why)
{
    if (batch.size() == 1) {
        end_request(s, batch[0], TS_ERR_CAPACITY, why);
    } else {
        for (size_t i = batch.size(); i-- > 0;) {
            batch[i]->state = RQ_QUEUED;
            batch[i]->requeued++;
            s->queue.push_front(batch[i]);
        }
        s->split_limit = std::max<size_t>(1, batch.size() / 2);
    }
    batch.clear();
    s->cv_done.notify_all();
}

void end_batch(Server *s, Slot &sl, ts_status st);
void try_admit(Server *s, Slot &sl);

// The count phase of a slot's batch completed: admit its rows (try_admit), or end the batch (no
// rows, an error), split it or grow its plan.
void count_done(Server *s, Slot &sl)
{
    ts_batch_status bs;
    ts_status st = plan_wait(sl.plan, &bs);
    if (st == TS_OK && bs.overflow) {
        // the batch outgrew the plan's tile or unit capacity: rebuild the plan at twice what the
        // device reported and run the batch again, unsplit
        BatchPlan *p = sl.plan;
        const uint64_t T = (uint64_t)p->h_out->hdr[HDR_T_LO] |
                           ((uint64_t)p->h_out->hdr[HDR_T_HI] << 32);
        uint64_t units = 0;
        if (p->b.quoff) {
            uint32_t u = 0;
            if (cudaMemcpy(&u, p->b.quoff + p->h_run[0], 4, cudaMemcpyDeviceToHost) == cudaSuccess)
                units = u;
            cudaGetLastError();
        }
        ts_batch_params bp = p->prm;
        bool grow = false;
        if (T > p->caps.tiles) {
            bp.max_tiles = 2 * T;
            grow = true;
        }
        if (units > p->caps.units) {
            bp.max_units = 2 * (uint64_t)units;
            bp.max_tiles = std::max<uint64_t>(bp.max_tiles, p->caps.tiles);
            grow = true;
        }
        BatchPlan *np = nullptr;
        if (grow && create_plan(p->ix, &bp, nullptr, false, &np) == TS_OK) {
            s->plan_bytes += np->dbytes;
            s->plan_bytes -= std::min(s->plan_bytes, (uint64_t)p->dbytes);
            destroy_plan(p);
            sl.plan = np;
            std::lock_guard<std::mutex> lk(s->mu);
            for (size_t i = sl.batch.size(); i-- > 0;) {
                sl.batch[i]->state = RQ_QUEUED;
                sl.batch[i]->requeued++;
                s->queue.push_front(sl.batch[i]);
            }
            sl.batch.clear();
            sl.busy = false;
            sl.phase = SLOT_IDLE;
            return;
        }
    }
    if (st == TS_OK && (bs.overflow || bs.rows > s->prm.max_batch_rows ||
                        ROW_BYTES * bs.rows > s->row_budget())) {
        std::lock_guard<std::mutex> lk(s->mu);
        split_batch(s, sl.batch, "request exceeds the server's per-batch row, memory or work "
                                 "capacity");
        sl.busy = false;
        sl.phase = SLOT_IDLE;
        return;
    }
    if (st == TS_OK && bs.rows > 0) {
        sl.rows = bs.rows;
        sl.phase = SLOT_ADMIT;
        sl.admit_since_us = s->now_us();
        try_admit(s, sl);
        return;
    }
    end_batch(s, sl, st);
}

// End a slot's batch without rows (none found, or a failure).
void end_batch(Server *s, Slot &sl, ts_status st)
{
    std::lock_guard<std::mutex> lk(s->mu);
    const char *msg = st == TS_OK ? nullptr : last_error();
    for (SrvReq *q : sl.batch) {
        q->out = SearchOut{};
        q->out.stats.n_queries = q->n;
        end_request(s, q, st, msg);
    }
    sl.batch.clear();
    sl.busy = false;
    sl.phase = SLOT_IDLE;
    if (st == TS_OK) s->split_limit = 0;
    s->cv_done.notify_all();
}

// Admission of a counted batch's rows: when they fit in the budget beside the rows still held
// (or nothing else is held), allocate them and launch the write phase; otherwise the slot stays
// in SLOT_ADMIT and the loop tries again. The budget is soft: after admit_wait_ms the batch is
// admitted beyond it if the device has the memory (the rows held may belong to results that
// completed but that the client has not collected yet, perhaps because it waits on this batch).
// An allocation that fails while other rows are held is retried until ten times that wait (at
// least 10 s), then the batch ends with TS_ERR_OOM; a stopping server cancels waiting batches.
void try_admit(Server *s, Slot &sl)
{
    if (s->stop) {
        set_error("server stopped before the batch's rows were admitted");
        end_batch(s, sl, TS_ERR_CANCELLED);
        return;
    }
    const uint64_t need = ROW_BYTES * sl.rows;
    const int64_t held = s->held->load();
    const double wait_ms = s->prm.admit_wait_ms ? (double)s->prm.admit_wait_ms : 1000.0;
    const double waited_ms = (s->now_us() - sl.admit_since_us) / 1e3;
    if (held > 0 && (uint64_t)held + need > s->row_budget() && waited_ms < wait_ms)
        return;  // wait for releases
    BatchPlan *p = sl.plan;
    auto block = std::make_shared<RowBlock>();
    block->held = s->held;
    ts_status st = block->alloc(sl.rows, p->stream);
    if (st == TS_ERR_OOM && held > 0 && waited_ms < std::max(10.0 * wait_ms, 10000.0)) {
        cudaGetLastError();
        return;  // retry after results are released
    }
    if (st == TS_OK) {
        p->b.out_q = block->q;
        p->b.out_e = block->e;
        p->b.out_tin = block->tin;
        p->b.out_tout = block->tout;
        p->caps.rows = sl.rows;
        st = pipe_write(p->ix, p->d_reqs, p->b, p->caps, p->stream);
    }
    if (st == TS_OK) {
        cudaError_t e = cudaMemcpyAsync(&p->h_out->status, p->b.status, 4,
                                        cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaEventRecord(sl.done, p->stream);
        if (e != cudaSuccess) st = cuda_status(e, "server write phase");
    }
    if (st == TS_OK) {
        sl.block = block;
        sl.phase = SLOT_WRITE;
        return;
    }
    end_batch(s, sl, st);
}

// The write phase of a slot's batch completed: every request gets a view of its rows.
void write_done(Server *s, Slot &sl)
{
    BatchPlan *p = sl.plan;
    ts_status st = TS_OK;
    cudaError_t e = cudaEventSynchronize(sl.done);
    if (e != cudaSuccess) st = cuda_status(e, "server write phase");
    if (st == TS_OK && p->h_out->status) st = read_dev_status(p->h_out->status);
    std::lock_guard<std::mutex> lk(s->mu);
    const char *msg = st == TS_OK ? nullptr : last_error();
    for (uint32_t r = 0; r < sl.batch.size(); r++) {
        SrvReq *q = sl.batch[r];
        if (st == TS_OK) {
            const uint64_t a = p->h_row0[r], n = p->h_row0[r + 1] - a;
            q->out = SearchOut{};
            q->out.count = n;
            q->out.stats.n_queries = q->n;
            q->out.stats.n_hits = n;
            if (n) {
                q->out.q = sl.block->q + a;
                q->out.e = sl.block->e + a;
                q->out.tin = sl.block->tin + a;
                q->out.tout = sl.block->tout + a;
                q->block = sl.block;
            }
        }
        end_request(s, q, st, msg);
    }
    sl.batch.clear();
    sl.block.reset();
    sl.busy = false;
    sl.phase = SLOT_IDLE;
    if (st == TS_OK) s->split_limit = 0;
    s->cv_done.notify_all();
}

// Form a batch for a free slot from the queue (caller holds the lock).
void form_batch(Server *s, std::vector<SrvReq *> &batch)
{
    const PipeCaps &k = s->slots[0].plan->caps;
    size_t limit = s->prm.max_batch_requests;
    if (s->split_limit) limit = std::min(limit, s->split_limit);
    uint64_t nq = 0;
    while (!s->queue.empty() && batch.size() < limit) {
        SrvReq *r = s->queue.front();
        if (r->n > k.nq) {  // can never fit
            s->queue.pop_front();
            end_request(s, r, TS_ERR_CAPACITY, "request has more query segments than a batch");
            s->cv_done.notify_all();
            continue;
        }
        if (nq + r->n > k.nq) break;
        s->queue.pop_front();
        nq += r->n;
        batch.push_back(r);
    }
}

ts_status launch_slot(Slot &sl)
{
    std::vector<ts_segments> segs(sl.batch.size());
    std::vector<ts_query_params> qps(sl.batch.size());
    for (size_t r = 0; r < sl.batch.size(); r++) {
        SrvReq *q = sl.batch[r];
        ts_segments &g = segs[r];
        memset(&g, 0, sizeof(g));
        const double *c = q->cols.data();
        g.x0 = c; g.y0 = c + q->n; g.z0 = c + 2 * q->n; g.t0 = c + 3 * q->n;
        g.x1 = c + 4 * q->n; g.y1 = c + 5 * q->n; g.z1 = c + 6 * q->n; g.t1 = c + 7 * q->n;
        g.n = q->n;
        g.on_host = 1;
        qps[r] = q->qp;
    }
    TS_CHECK(plan_run(sl.plan, (uint32_t)sl.batch.size(), segs.data(), qps.data(), nullptr));
    TS_CUDA(cudaEventRecord(sl.done, sl.plan->stream));
    sl.phase = SLOT_COUNT;
    return TS_OK;
}

void loop(Server *s)
{
    cudaSetDevice(s->device);
    constexpr double SPIN_US = 2000.0;  // poll without sleeping this long after any progress
    double spin_until = 0.0;
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool any_busy = false;
        for (Slot &sl : s->slots) any_busy = any_busy || sl.busy;
        if (s->stop && !any_busy) break;
        // completions
        bool progressed = false;
        for (Slot &sl : s->slots) {
            if (!sl.busy) continue;
            if (sl.phase == SLOT_ADMIT) {  // waiting for room for its rows
                lk.unlock();
                try_admit(s, sl);
                lk.lock();
                progressed = progressed || sl.phase != SLOT_ADMIT;
                continue;
            }
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            lk.unlock();
            if (sl.phase == SLOT_COUNT) count_done(s, sl); else write_done(s, sl);
            lk.lock();
            progressed = true;
        }
        // launches
        for (Slot &sl : s->slots) {
            if (sl.busy || s->stop || s->queue.empty()) continue;
            bool others_busy = false;
            for (Slot &o : s->slots) others_busy = others_busy || (&o != &sl && o.busy);
            // linger: a partly filled batch waits briefly while another batch is on the device
            if (others_busy && s->queue.size() < s->prm.max_batch_requests &&
                s->now_us() - s->queue.front()->submit_us < (double)s->prm.linger_us)
                continue;
            form_batch(s, sl.batch);
            if (sl.batch.empty()) continue;
            const double t = s->now_us();
            for (SrvReq *q : sl.batch) {
                q->state = RQ_RUNNING;
                q->start_us = t;
                q->batch_requests = (uint32_t)sl.batch.size();
            }
            lk.unlock();
            ts_status st = launch_slot(sl);
            lk.lock();
            if (st != TS_OK) {
                const char *msg = last_error();
                for (SrvReq *q : sl.batch) end_request(s, q, st, msg);
                sl.batch.clear();
                s->cv_done.notify_all();
                continue;
            }
            sl.busy = true;
            progressed = true;
        }
        if (progressed) {
            spin_until = s->now_us() + SPIN_US;
            continue;
        }
        any_busy = false;
        for (Slot &sl : s->slots) any_busy = any_busy || sl.busy;
        if (any_busy) {
            // a batch is on the device: poll its completion, yielding the core (a sleep of a few
            // microseconds oversleeps by tens), and sleeping only once nothing has progressed
            // for SPIN_US
            lk.unlock();
            if (s->now_us() < spin_until)
                std::this_thread::yield();
            else
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
    // queued requests left at stop are cancelled
    while (!s->queue.empty()) {
        SrvReq *r = s->queue.front();
        s->queue.pop_front();
        end_request(s, r, TS_ERR_CANCELLED, "server stopped");
    }
    s->cv_done.notify_all();
}

}  // namespace

ts_status server_create(const Index *ix, const ts_server_params *prm, Server **out)
{
    *out = nullptr;
    if (!prm || prm->max_batch_requests == 0 || prm->max_batch_queries == 0 ||
        prm->max_batch_rows == 0) {
        set_error("ts_server_create: need max_batch_requests, max_batch_queries, max_batch_rows");
        return TS_ERR_INVALID_ARG;
    }
    std::unique_ptr<Server> s(new Server());
    s->ix = ix;
    s->prm = *prm;
    if (s->prm.max_inflight == 0) s->prm.max_inflight = 2;
    TS_CUDA(cudaGetDevice(&s->device));
    s->budget = prm->mem_budget_bytes;
    if (!s->budget) {
        // three quarters of the device memory free once the pool's unused blocks are returned
        pool_trim();
        size_t free_b = 0, total_b = 0;
        TS_CUDA(cudaMemGetInfo(&free_b, &total_b));
        s->budget = free_b / 4 * 3;
    }
    s->slots.resize(s->prm.max_inflight);
    ts_batch_params bp;
    memset(&bp, 0, sizeof(bp));
    bp.max_requests = prm->max_batch_requests;
    bp.max_queries = prm->max_batch_queries;
    bp.tile_records = prm->tile_records;
    bp.use_graph = prm->use_graph;
    // hits a batch's count pass keeps: an eighth of the budget per plan (32 B per hit)
    bp.scratch_rows = prm->scratch_rows
                          ? prm->scratch_rows
                          : std::max<uint64_t>(1ull << 20, s->budget / 8 / 32);
    for (Slot &sl : s->slots) {
        // the plans run up to the row scan; every batch's rows are allocated at its exact size
        ts_status st = create_plan(ix, &bp, nullptr, false, &sl.plan);
        if (st == TS_OK) s->plan_bytes += sl.plan->dbytes;
        if (st == TS_OK) {
            cudaError_t e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
            if (e != cudaSuccess) st = cuda_status(e, "cudaEventCreate(server)");
        }
        if (st != TS_OK) {
            for (Slot &o : s->slots) {
                if (o.plan) destroy_plan(o.plan);
                if (o.done) cudaEventDestroy(o.done);
            }
            return st;
        }
    }
    s->t0 = std::chrono::steady_clock::now();
    Server *raw = s.release();
    raw->th = std::thread(loop, raw);
    *out = raw;
    return TS_OK;
}

ts_status server_submit(Server *s, const ts_segments *q, const ts_query_params *qp,
                        uint64_t *ticket)
{
    if (!q || !ticket) {
        set_error("ts_server_submit: NULL argument");
        return TS_ERR_INVALID_ARG;
    }
    TS_CHECK(check_query_params(qp));
    std::unique_ptr<SrvReq> r(new SrvReq());
    r->n = q->n;
    r->qp = *qp;
    r->cols.resize(8 * q->n);
    const double *src[8] = {q->x0, q->y0, q->z0, q->t0, q->x1, q->y1, q->z1, q->t1};
    for (int c = 0; c < 8; c++) {
        if (!q->n) break;
        if (!src[c]) {
            set_error("ts_server_submit: NULL column %d", c);
            return TS_ERR_INVALID_ARG;
        }
        if (q->on_host) {
            memcpy(r->cols.data() + (uint64_t)c * q->n, src[c], 8 * q->n);
        } else {
            TS_CUDA(cudaMemcpy(r->cols.data() + (uint64_t)c * q->n, src[c], 8 * q->n,
                               cudaMemcpyDeviceToHost));
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        set_error("ts_server_submit: server is stopping");
        return TS_ERR_CANCELLED;
    }
    r->ticket = s->next_ticket++;
    r->submit_us = s->now_us();
    *ticket = r->ticket;
    s->reqs[r->ticket] = r.get();
    s->queue.push_back(r.release());
    s->cv_work.notify_one();
    return TS_OK;
}

ts_status server_wait(Server *s, uint64_t ticket, uint32_t timeout_ms, SearchOut *out,
                      std::shared_ptr<RowBlock> *block, ts_request_timing *timing)
{
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("ts_server_wait: unknown ticket %llu", (unsigned long long)ticket);
        return TS_ERR_INVALID_ARG;
    }
    SrvReq *r = it->second;
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return r->state == RQ_DONE; });
    if (!ok) {
        set_error("ts_server_wait: request %llu not done within %u ms",
                  (unsigned long long)ticket, timeout_ms);
        return TS_ERR_TIMEOUT;
    }
    s->reqs.erase(it);
    if (timing) {
        timing->submit_us = r->submit_us;
        timing->start_us = r->start_us;
        timing->done_us = r->done_us;
        timing->batch_requests = r->batch_requests;
        timing->requeued = r->requeued;
    }
    const ts_status st = r->status;
    if (st == TS_OK) {
        *out = r->out;
        if (block) *block = r->block;
        r->out = SearchOut{};
    } else {
        set_error("%s", r->error.c_str());
    }
    delete r;
    return st;
}

void server_info(Server *s, uint64_t *budget, uint64_t *plan_bytes, uint64_t *held_bytes)
{
    std::lock_guard<std::mutex> lk(s->mu);
    if (budget) *budget = s->budget;
    if (plan_bytes) *plan_bytes = s->plan_bytes;
    if (held_bytes) {
        const int64_t h = s->held->load();
        *held_bytes = h > 0 ? (uint64_t)h : 0;
    }
}

ts_status server_cancel(Server *s, uint64_t ticket)
{
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second->state != RQ_QUEUED) {
        set_error("ts_server_cancel: request %llu is not queued", (unsigned long long)ticket);
        return TS_ERR_INVALID_ARG;
    }
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
        if (*q == it->second) {
            s->queue.erase(q);
            break;
        }
    end_request(s, it->second, TS_ERR_CANCELLED, "cancelled");
    s->cv_done.notify_all();
    return TS_OK;
}

void server_destroy(Server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    for (auto &kv : s->reqs) delete kv.second;  // (undelivered rows go with their block)
    for (Slot &sl : s->slots) {
        if (sl.plan) destroy_plan(sl.plan);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    s->magic = 0;
    delete s;
}

}  // namespace ts
