// ts_server.cu -- the served search: a request loop on a resident index with continuous batching.
//
// Client threads submit requests (their query segments are copied into the request); one loop
// thread forms batches from the queue in arrival order while a batch's request, query and row
// capacities allow, and runs them on up to max_inflight batch plans, each with its own stream:
// requests that arrive while a batch is on the device go into the next free plan, so batches
// overlap on the device. A batch whose rows overflow is split and re-run; a lone request that
// cannot fit ends with TS_ERR_CAPACITY. Completed requests get their own device rows (copied out
// of the plan) and host timestamps. Every wait -- client waits and the loop's idle waits -- is
// bounded.
#include <string.h>

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
    int state = RQ_QUEUED;
    ts_status status = TS_OK;
    std::string error;
    SearchOut out;
};

struct Slot {
    BatchPlan *plan = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<SrvReq *> batch;
    bool busy = false;
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
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t split_limit = 0;  // after an overflow: at most this many requests in the next batch
    std::chrono::steady_clock::time_point t0;

    double now_us() const
    {
        return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0)
            .count();
    }
};

namespace {

void free_out(SearchOut &o)
{
    if (o.q) cudaFreeAsync(o.q, 0);
    if (o.e) cudaFreeAsync(o.e, 0);
    if (o.tin) cudaFreeAsync(o.tin, 0);
    if (o.tout) cudaFreeAsync(o.tout, 0);
    o = SearchOut{};
}

void end_request(Server *s, SrvReq *r, ts_status st, const char *msg)
{
    r->status = st;
    if (msg) r->error = msg;
    r->state = RQ_DONE;
    r->done_us = s->now_us();
}

// Copy a request's rows out of the plan into its own device arrays.
ts_status take_rows(BatchPlan *p, uint32_t r, SrvReq *q)
{
    uint64_t first = 0, count = 0;
    TS_CHECK(plan_request_rows(p, r, &first, &count));
    q->out.count = count;
    q->out.stats.n_queries = q->n;
    q->out.stats.n_hits = count;
    if (!count) return TS_OK;
    cudaStream_t st = p->stream;
    TS_CUDA(pool_malloc((void **)&q->out.q, 4 * count, st));
    TS_CUDA(pool_malloc((void **)&q->out.e, 4 * count, st));
    TS_CUDA(pool_malloc((void **)&q->out.tin, 8 * count, st));
    TS_CUDA(pool_malloc((void **)&q->out.tout, 8 * count, st));
    TS_CUDA(cudaMemcpyAsync(q->out.q, p->b.out_q + first, 4 * count, cudaMemcpyDeviceToDevice, st));
    TS_CUDA(cudaMemcpyAsync(q->out.e, p->b.out_e + first, 4 * count, cudaMemcpyDeviceToDevice, st));
    TS_CUDA(cudaMemcpyAsync(q->out.tin, p->b.out_tin + first, 8 * count, cudaMemcpyDeviceToDevice, st));
    TS_CUDA(cudaMemcpyAsync(q->out.tout, p->b.out_tout + first, 8 * count, cudaMemcpyDeviceToDevice, st));
    return TS_OK;
}

// Called by the loop when a slot's batch has completed on the device.
void finish_slot(Server *s, Slot &sl)
{
    ts_batch_status bs;
    ts_status st = plan_wait(sl.plan, &bs);
    std::vector<SrvReq *> batch;
    batch.swap(sl.batch);
    sl.busy = false;
    if (st == TS_OK && bs.overflow) {
        std::lock_guard<std::mutex> lk(s->mu);
        if (batch.size() == 1) {
            end_request(s, batch[0], TS_ERR_CAPACITY,
                        "request exceeds the server's per-batch row or work capacity");
        } else {
            // re-queue at the front, in order; the next batches take half as many requests
            for (size_t i = batch.size(); i-- > 0;) {
                batch[i]->state = RQ_QUEUED;
                s->queue.push_front(batch[i]);
            }
            s->split_limit = std::max<size_t>(1, batch.size() / 2);
        }
        s->cv_done.notify_all();
        return;
    }
    if (st == TS_OK) {
        for (uint32_t r = 0; r < batch.size() && st == TS_OK; r++) st = take_rows(sl.plan, r, batch[r]);
        if (st == TS_OK) {
            cudaError_t e = cudaStreamSynchronize(sl.plan->stream);
            if (e != cudaSuccess) st = cuda_status(e, "cudaStreamSynchronize(server)");
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    const char *msg = st == TS_OK ? nullptr : last_error();
    for (SrvReq *q : batch) {
        if (st != TS_OK) free_out(q->out);
        end_request(s, q, st, msg);
    }
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

ts_status launch_slot(Server *s, Slot &sl)
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
    return TS_OK;
}

void loop(Server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool any_busy = false;
        for (Slot &sl : s->slots) any_busy = any_busy || sl.busy;
        if (s->stop && !any_busy) break;
        // completions
        bool progressed = false;
        for (Slot &sl : s->slots) {
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            lk.unlock();
            finish_slot(s, sl);
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
            ts_status st = launch_slot(s, sl);
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
        if (progressed) continue;
        any_busy = false;
        for (Slot &sl : s->slots) any_busy = any_busy || sl.busy;
        if (any_busy) {
            // a batch is on the device: poll its completion at a short period
            lk.unlock();
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
    s->slots.resize(s->prm.max_inflight);
    ts_batch_params bp;
    memset(&bp, 0, sizeof(bp));
    bp.max_requests = prm->max_batch_requests;
    bp.max_queries = prm->max_batch_queries;
    bp.max_rows = prm->max_batch_rows;
    bp.tile_records = prm->tile_records;
    bp.use_graph = prm->use_graph;
    for (Slot &sl : s->slots) {
        ts_status st = create_plan(ix, &bp, nullptr, true, &sl.plan);
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
                      ts_request_timing *timing)
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
        timing->reserved = 0;
    }
    const ts_status st = r->status;
    if (st == TS_OK) {
        *out = r->out;
        r->out = SearchOut{};
    } else {
        set_error("%s", r->error.c_str());
        free_out(r->out);
    }
    delete r;
    return st;
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
    for (auto &kv : s->reqs) {
        free_out(kv.second->out);
        delete kv.second;
    }
    for (Slot &sl : s->slots) {
        if (sl.plan) destroy_plan(sl.plan);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    s->magic = 0;
    delete s;
}

}  // namespace ts
