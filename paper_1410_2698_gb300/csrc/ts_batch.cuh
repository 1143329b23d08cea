// ts_batch.cuh -- batch plans (reusable pipelines with fixed capacities) and shared row blocks.
#pragma once

#include <atomic>
#include <memory>
#include <vector>

#include "ts_search.cuh"

namespace ts {

constexpr uint32_t MAGIC_BATCH = 0x54534254u;  // "TSBT"

// Outcome of a run, written by the device into mapped pinned memory.
struct BatchOut {
    uint32_t hdr[8];
    unsigned long long stats[ST_NSLOTS];
    uint32_t status;
    uint32_t pad[3];
};

struct BatchPlan {
    uint32_t magic = MAGIC_BATCH;
    const Index *ix = nullptr;
    ts_batch_params prm{};
    PipeCaps caps;
    PipeBufs b{};
    bool own_rows = true;
    // device memory (one allocation)
    void *dmem = nullptr;
    size_t dbytes = 0;
    ReqDesc *d_reqs = nullptr;
    uint32_t *d_run = nullptr;
    // mapped pinned host memory (one allocation)
    void *hmem = nullptr;
    size_t hbytes = 0;
    ReqDesc *h_reqs = nullptr;
    uint32_t *h_run = nullptr;
    double *h_stage = nullptr;
    BatchOut *h_out = nullptr;
    unsigned long long *h_row0 = nullptr;
    // the same mapped pinned memory as device pointers
    ReqDesc *dh_reqs = nullptr;
    uint32_t *dh_run = nullptr;
    BatchOut *dh_out = nullptr;
    unsigned long long *dh_row0 = nullptr;
    double *dh_stage = nullptr;
    // execution
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long graph_kernels = 0;  // kernel launches captured in the graph
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // count pass, write pass bounds
    // recorded after each run on the stream it ran on: waiting for a run, and copying its rows
    // on the plan's own stream, need not wait for later work on a stream the plan shares
    cudaEvent_t done = nullptr;
    bool running = false;
    uint32_t last_nreq = 0;
};

// Device rows shared by the results of a one-shot batch or a served batch. `held`, when set,
// counts the bytes of live row blocks (the served loop's admission): alloc adds the block's
// bytes, the destructor (when the last result using the rows is released) subtracts them.
struct RowBlock {
    uint32_t *q = nullptr, *e = nullptr;
    double *tin = nullptr, *tout = nullptr;
    std::shared_ptr<std::atomic<int64_t>> held;
    uint64_t bytes = 0;
    ts_status alloc(uint64_t n, cudaStream_t s);
    ~RowBlock();
};
constexpr uint64_t ROW_BYTES = 2 * sizeof(uint32_t) + 2 * sizeof(double);

void note_launches(unsigned long long n);

ts_status create_plan(const Index *ix, const ts_batch_params *prm, cudaStream_t s, bool own_rows,
                      BatchPlan **out);
void destroy_plan(BatchPlan *p);
ts_status plan_run(BatchPlan *p, uint32_t nreq, const ts_segments *qs, const ts_query_params *qps,
                   cudaStream_t s);
ts_status plan_wait(BatchPlan *p, ts_batch_status *out);
ts_status plan_request_rows(const BatchPlan *p, uint32_t r, uint64_t *first, uint64_t *count);
ts_status search_batch(const Index *ix, uint32_t nreq, const ts_segments *qs,
                       const ts_query_params *qps, cudaStream_t s,
                       std::vector<SearchOut> &outs, std::shared_ptr<RowBlock> &block);

}  // namespace ts
