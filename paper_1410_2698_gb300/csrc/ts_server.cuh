// ts_server.cuh -- the served search (request loop with continuous batching).
#pragma once

#include <memory>

#include "ts_batch.cuh"

namespace ts {

constexpr uint32_t MAGIC_SERVER = 0x54535356u;  // "TSSV"

struct Server;

ts_status server_create(const Index *ix, const ts_server_params *prm, Server **out);
ts_status server_submit(Server *s, const ts_segments *q, const ts_query_params *qp,
                        uint64_t *ticket);
ts_status server_wait(Server *s, uint64_t ticket, uint32_t timeout_ms, SearchOut *out,
                      std::shared_ptr<RowBlock> *block, ts_request_timing *timing);
ts_status server_cancel(Server *s, uint64_t ticket);
void server_info(Server *s, uint64_t *budget, uint64_t *plan_bytes, uint64_t *held_bytes);
void server_destroy(Server *s);

}  // namespace ts
