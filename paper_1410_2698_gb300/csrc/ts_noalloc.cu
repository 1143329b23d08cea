// ts_noalloc.cu -- an all-pairs search that allocates no memory.
//
// Who this is for: code that runs inside a host application which owns every byte of device
// memory through its own allocator or a fixed budget (a library-side cudaMalloc would bypass that
// accounting or fail), and latency-sensitive callers for whom cudaMalloc/cudaFree, which can
// synchronise the device, are not acceptable on the request path. Such callers pass their input
// and output arrays; the only working memory is TS_NOALLOC_SCRATCH_BYTES of device memory that is
// part of this library's image (a file-scope __device__ array), which every GPU that loads the
// library holds until the process exits.
//
// Work layout: tiles of 32 query segments x 1024 database segments in the caller's order; pass 1
// counts each tile's hits into the scratch array, a three-kernel scan turns the counts into row
// offsets (also in the scratch array), pass 2 writes the rows. The pair test is the same three-
// stage test as the indexed search (FP32 box filter, FP32 gap filter, exact FP64 closed form).
#include <mutex>

#include "ts_device.cuh"

namespace ts {

namespace {

constexpr uint64_t NA_SCRATCH_BYTES = 32ull << 20;  // TS_NOALLOC_SCRATCH_BYTES
constexpr int NA_QB = 32;                           // query segments per tile
constexpr int NA_EB = 1024;                         // database segments per tile
constexpr int NA_SCAN = 2048;                       // tiles per scan block
constexpr uint64_t NA_MAX_TILES = 2500000;          // TS_NOALLOC_MAX_TILES
constexpr uint64_t NA_CTRL = 256;
constexpr uint64_t NA_COUNTS = NA_CTRL;
constexpr uint64_t NA_OFFS = (NA_COUNTS + 4 * NA_MAX_TILES + 255) / 256 * 256;
constexpr uint64_t NA_PARTS = (NA_OFFS + 8 * (NA_MAX_TILES + 1) + 255) / 256 * 256;
constexpr uint64_t NA_MAX_PARTS = (NA_MAX_TILES + NA_SCAN - 1) / NA_SCAN;
static_assert(NA_PARTS + 8 * (NA_MAX_PARTS + 1) <= NA_SCRATCH_BYTES, "scratch layout");
static_assert(NA_MAX_PARTS <= 2048, "one block scans the partial sums");

// The scratch: shared by every call of ts_search_brute_noalloc on a device.
static __device__ __align__(256) unsigned char g_na_scratch[NA_SCRATCH_BYTES];

struct NaCtrl {
    uint32_t status;
    uint32_t pad[3];
    unsigned long long total;
};

struct NaParams {
    const double *e[8];
    const double *q[8];
    uint64_t n, nq;
    uint64_t nchunk, ntiles;
    double d, dd, Ts, Te;
    float d_up, d2u;
    uint32_t *q_out, *e_out;
    double *tin_out, *tout_out;
    unsigned char *scratch;  // device address of g_na_scratch
};

struct NaMember {
    QueryD q;
    float4 ea, eb, ua, ub;
    uint32_t live;
    uint32_t pad[3];
};

constexpr int NA_WARPS = 8;

template <int PASS>
__global__ void __launch_bounds__(NA_WARPS * 32) k_na_tiles(NaParams P)
{
    __shared__ NaMember mem[NA_WARPS][NA_QB];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu;
    const uint32_t lt_mask = (1u << lane) - 1u;
    NaCtrl *ctrl = reinterpret_cast<NaCtrl *>(P.scratch);
    uint32_t *counts = reinterpret_cast<uint32_t *>(P.scratch + NA_COUNTS);
    const unsigned long long *offs = reinterpret_cast<const unsigned long long *>(P.scratch + NA_OFFS);
    const uint64_t nwarps = (uint64_t)gridDim.x * NA_WARPS;
    for (uint64_t t = (uint64_t)blockIdx.x * NA_WARPS + wid; t < P.ntiles; t += nwarps) {
        const uint64_t qb = t / P.nchunk, ch = t % P.nchunk;
        const uint64_t q0 = qb * NA_QB, e0 = ch * NA_EB;
        const uint32_t nmem = (uint32_t)((P.nq - q0) < NA_QB ? (P.nq - q0) : NA_QB);
        const uint32_t nent = (uint32_t)((P.n - e0) < NA_EB ? (P.n - e0) : NA_EB);
        // members: the tile's query segments
        if ((uint32_t)lane < nmem) {
            const uint64_t i = q0 + lane;
            double v[8];
            bool fin = true;
            for (int k = 0; k < 8; k++) {
                v[k] = P.q[k][i];
                fin = fin && isfinite(v[k]);
            }
            if (!fin || !(v[7] > v[3])) atomicOr(&ctrl->status, DEV_ERR_INVALID);
            const double dt = v[7] - v[3];
            NaMember &M = mem[wid][lane];
            M.q.vx = (v[4] - v[0]) / dt;
            M.q.vy = (v[5] - v[1]) / dt;
            M.q.vz = (v[6] - v[2]) / dt;
            M.q.w0 = dmx(v[3], P.Ts);
            M.q.w1 = dmn(v[7], P.Te);
            const double dw = M.q.w0 - v[3];  // 0 unless the request interval clips the start
            M.q.xw = fma(M.q.vx, dw, v[0]);
            M.q.yw = fma(M.q.vy, dw, v[1]);
            M.q.zw = fma(M.q.vz, dw, v[2]);
            M.q.ndd = -P.dd;
            M.q.pad = 0.0;
            float mn[3], mx[3];
            for (int d = 0; d < 3; d++) {
                mn[d] = __double2float_rd(v[d] < v[4 + d] ? v[d] : v[4 + d]);
                mx[d] = __double2float_ru(v[d] < v[4 + d] ? v[4 + d] : v[d]);
            }
            M.ea = make_float4(__fsub_rd(mn[0], P.d_up), __fsub_rd(mn[1], P.d_up),
                               __fsub_rd(mn[2], P.d_up), __double2float_rd(M.q.w0));
            M.eb = make_float4(__fadd_ru(mx[0], P.d_up), __fadd_ru(mx[1], P.d_up),
                               __fadd_ru(mx[2], P.d_up), __double2float_ru(M.q.w1));
            M.ua = make_float4(mn[0], mn[1], mn[2], P.d2u);
            M.ub = make_float4(mx[0], mx[1], mx[2], 0.0f);
            M.live = (fin && v[7] > v[3] && M.q.w0 < M.q.w1) ? 1u : 0u;
        }
        __syncwarp();
        uint64_t hits = 0;
        const uint64_t wbase = PASS == 1 ? offs[t] : 0;
        const uint64_t wend = PASS == 1 ? offs[t + 1] : 0;
        for (uint32_t bb = 0; bb < nent; bb += 32) {
            const uint32_t j = bb + lane;
            const bool inb = j < nent;
            const uint64_t ei = e0 + (inb ? j : 0);
            double v[8];
            bool fin = true;
            for (int k = 0; k < 8; k++) {
                v[k] = P.e[k][ei];
                fin = fin && isfinite(v[k]);
            }
            if (inb && (!fin || !(v[7] > v[3]))) atomicOr(&ctrl->status, DEV_ERR_INVALID);
            const double dt = v[7] - v[3];
            SegD e;
            e.x0 = v[0]; e.y0 = v[1]; e.z0 = v[2]; e.t0 = v[3]; e.t1 = v[7];
            e.vx = (v[4] - v[0]) / dt;
            e.vy = (v[5] - v[1]) / dt;
            e.vz = (v[6] - v[2]) / dt;
            RecF r;
            r.xmin = __double2float_rd(fmin(v[0], v[4])); r.xmax = __double2float_ru(fmax(v[0], v[4]));
            r.ymin = __double2float_rd(fmin(v[1], v[5])); r.ymax = __double2float_ru(fmax(v[1], v[5]));
            r.zmin = __double2float_rd(fmin(v[2], v[6])); r.zmax = __double2float_ru(fmax(v[2], v[6]));
            r.t0 = __double2float_rd(v[3]);
            r.t1 = __double2float_ru(v[7]);
            const bool use = inb && fin && (v[7] > v[3]);
            for (uint32_t m = 0; m < nmem; m++) {
                const NaMember &M = mem[wid][m];
                if (!M.live) continue;  // warp-uniform
                bool p = use && filter_box(r, M.ea, M.eb) && filter_gap(r, M.ua, M.ub);
                bool h = false;
                double tin = 0.0, tout = 0.0;
                if (p) {
                    Quad qd;
                    h = pair_quad(M.q, e, qd) && quad_solve(qd, PASS == 1, &tin, &tout);
                }
                const unsigned hm = __ballot_sync(FULL, h);
                if (PASS == 1 && h) {
                    const uint64_t o = wbase + hits + __popc(hm & lt_mask);
                    if (o < wend) {
                        P.q_out[o] = (uint32_t)(q0 + m);
                        P.e_out[o] = (uint32_t)(e0 + j);
                        P.tin_out[o] = tin;
                        P.tout_out[o] = tout;
                    }
                }
                hits += __popc(hm);
            }
        }
        if (PASS == 0) {
            if (lane == 0) {
                if (hits > 0xffffffffull) atomicOr(&ctrl->status, DEV_ERR_OVERFLOW);
                counts[t] = (uint32_t)hits;
            }
        } else {
            if (lane == 0 && wbase + hits != wend) atomicOr(&ctrl->status, DEV_ERR_INTERNAL);
        }
        __syncwarp();
    }
}

// Scan of the tile counts into row offsets, in three launches that use only the scratch array.
__device__ __forceinline__ unsigned long long na_block_scan(unsigned long long v,
                                                            unsigned long long *total)
{
    __shared__ unsigned long long ws[33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = lane < nw ? ws[lane] : 0ull;
        unsigned long long wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) ws[lane] = wi - w;
        if (lane == 31) ws[32] = wi;
    }
    __syncthreads();
    const unsigned long long r = ws[wid] + x - v;
    *total = ws[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(1024) k_na_scan_parts(unsigned char *scratch, uint64_t ntiles)
{
    const uint32_t *counts = reinterpret_cast<const uint32_t *>(scratch + NA_COUNTS);
    unsigned long long *parts = reinterpret_cast<unsigned long long *>(scratch + NA_PARTS);
    unsigned long long s = 0;
    const uint64_t base = (uint64_t)blockIdx.x * NA_SCAN;
    for (uint64_t k = threadIdx.x; k < NA_SCAN; k += blockDim.x)
        if (base + k < ntiles) s += counts[base + k];
    unsigned long long tot;
    na_block_scan(s, &tot);
    if (threadIdx.x == 0) parts[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_na_scan_top(unsigned char *scratch, uint64_t nparts)
{
    unsigned long long *parts = reinterpret_cast<unsigned long long *>(scratch + NA_PARTS);
    NaCtrl *ctrl = reinterpret_cast<NaCtrl *>(scratch);
    // two parts per thread, in order
    const uint64_t a = 2 * threadIdx.x, b = a + 1;
    const unsigned long long va = a < nparts ? parts[a] : 0ull, vb = b < nparts ? parts[b] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = na_block_scan(va + vb, &tot);
    if (a < nparts) parts[a] = ex;
    if (b < nparts) parts[b] = ex + va;
    if (threadIdx.x == 0) ctrl->total = tot;
}

__global__ void __launch_bounds__(1024) k_na_scan_final(unsigned char *scratch, uint64_t ntiles)
{
    const uint32_t *counts = reinterpret_cast<const uint32_t *>(scratch + NA_COUNTS);
    unsigned long long *offs = reinterpret_cast<unsigned long long *>(scratch + NA_OFFS);
    const unsigned long long *parts = reinterpret_cast<const unsigned long long *>(scratch + NA_PARTS);
    const NaCtrl *ctrl = reinterpret_cast<const NaCtrl *>(scratch);
    const uint64_t base = (uint64_t)blockIdx.x * NA_SCAN;
    // two consecutive tiles per thread
    const uint64_t a = base + 2 * threadIdx.x, b = a + 1;
    const unsigned long long va = a < ntiles ? counts[a] : 0ull, vb = b < ntiles ? counts[b] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = parts[blockIdx.x] + na_block_scan(va + vb, &tot);
    if (a < ntiles) offs[a] = ex;
    if (b < ntiles) offs[b] = ex + va;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) offs[ntiles] = ctrl->total;
}

// Device address of g_na_scratch per device, looked up once per device (with that device
// current) on the first call that runs on it.
std::mutex g_na_mu;
unsigned char *g_na_ptr[256] = {nullptr};

ts_status na_scratch(unsigned char **out)
{
    int dev = 0;
    TS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        set_error("ts_search_brute_noalloc: device ordinal %d out of range", dev);
        return TS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) return cuda_status(e, "cudaGetSymbolAddress(g_na_scratch)");
        g_na_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_na_ptr[dev];
    return TS_OK;
}

float na_float_up(double x)
{
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}

ts_status na_status(uint32_t st)
{
    if (st & DEV_ERR_INVALID) {
        set_error("invalid segment (NaN/Inf or t_end <= t_start)");
        return TS_ERR_INVALID_ARG;
    }
    if (st & DEV_ERR_OVERFLOW) {
        set_error("a tile's hit count does not fit in 32 bits");
        return TS_ERR_CAPACITY;
    }
    if (st) {
        set_error("no-allocation search: device status 0x%x", st);
        return TS_ERR_INTERNAL;
    }
    return TS_OK;
}

}  // namespace

ts_status search_brute_noalloc(const ts_segments *db, const ts_segments *q,
                               const ts_query_params *qp, uint32_t *q_idx, uint32_t *e_idx,
                               double *t_in, double *t_out, uint64_t capacity, uint64_t *count,
                               cudaStream_t s)
{
    if (!db || !q || !qp || !count) {
        set_error("ts_search_brute_noalloc: NULL argument");
        return TS_ERR_INVALID_ARG;
    }
    *count = 0;
    if (db->on_host || q->on_host) {
        set_error("ts_search_brute_noalloc: inputs must be device pointers (on_host = 0)");
        return TS_ERR_INVALID_ARG;
    }
    if (!(qp->d > 0.0) || !isfinite(qp->d) || isnan(qp->t_start) || isnan(qp->t_end) ||
        qp->t_start > qp->t_end) {
        set_error("ts_search_brute_noalloc: need finite d > 0 and t_start <= t_end");
        return TS_ERR_INVALID_ARG;
    }
    if (db->n > 0xffffffffull || q->n > 0xffffffffull) {
        set_error("ts_search_brute_noalloc: sizes above 2^32 - 1");
        return TS_ERR_INVALID_ARG;
    }
    const double *ec[8] = {db->x0, db->y0, db->z0, db->t0, db->x1, db->y1, db->z1, db->t1};
    const double *qc[8] = {q->x0, q->y0, q->z0, q->t0, q->x1, q->y1, q->z1, q->t1};
    for (int k = 0; k < 8; k++)
        if ((db->n && !ec[k]) || (q->n && !qc[k])) {
            set_error("ts_search_brute_noalloc: NULL column %d", k);
            return TS_ERR_INVALID_ARG;
        }
    if (db->n == 0 || q->n == 0) return TS_OK;
    const uint64_t nchunk = (db->n + NA_EB - 1) / NA_EB;
    const uint64_t ntiles = (q->n + NA_QB - 1) / NA_QB * nchunk;
    if (ntiles > NA_MAX_TILES) {
        set_error("ts_search_brute_noalloc: %llu tiles of 32 query x 1024 database segments "
                  "exceed the fixed scratch limit of %llu tiles",
                  (unsigned long long)ntiles, (unsigned long long)NA_MAX_TILES);
        return TS_ERR_CAPACITY;
    }
    unsigned char *scratch = nullptr;
    TS_CHECK(na_scratch(&scratch));
    NaParams P;
    for (int k = 0; k < 8; k++) {
        P.e[k] = ec[k];
        P.q[k] = qc[k];
    }
    P.n = db->n;
    P.nq = q->n;
    P.nchunk = nchunk;
    P.ntiles = ntiles;
    P.d = qp->d;
    P.dd = qp->d * qp->d;
    P.Ts = qp->t_start;
    P.Te = qp->t_end;
    P.d_up = na_float_up(qp->d);
    P.d2u = na_float_up(P.dd * (1.0 + 1e-6));
    P.q_out = q_idx;
    P.e_out = e_idx;
    P.tin_out = t_in;
    P.tout_out = t_out;
    P.scratch = scratch;
    int dev = 0, sms = 0;
    TS_CUDA(cudaGetDevice(&dev));
    TS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint64_t want = (ntiles + NA_WARPS - 1) / NA_WARPS;
    const unsigned grid = (unsigned)(want < (uint64_t)sms * 4 ? want : (uint64_t)sms * 4);
    const uint64_t nparts = (ntiles + NA_SCAN - 1) / NA_SCAN;

    // the control words start at zero on every call; counts and offsets are fully rewritten
    TS_CUDA(cudaMemsetAsync(scratch, 0, NA_CTRL, s));
    k_na_tiles<0><<<grid, NA_WARPS * 32, 0, s>>>(P);
    TS_LAUNCHED();
    k_na_scan_parts<<<(unsigned)nparts, 1024, 0, s>>>(scratch, ntiles);
    TS_LAUNCHED();
    k_na_scan_top<<<1, 1024, 0, s>>>(scratch, nparts);
    TS_LAUNCHED();
    k_na_scan_final<<<(unsigned)nparts, 1024, 0, s>>>(scratch, ntiles);
    TS_LAUNCHED();
    NaCtrl h;
    TS_CUDA(cudaMemcpyAsync(&h, scratch, sizeof(NaCtrl), cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaStreamSynchronize(s));
    TS_CHECK(na_status(h.status));
    *count = h.total;
    if (h.total > capacity) {
        set_error("ts_search_brute_noalloc: %llu result rows exceed the capacity %llu",
                  (unsigned long long)h.total, (unsigned long long)capacity);
        return TS_ERR_CAPACITY;
    }
    if (h.total == 0) return TS_OK;
    if (!q_idx || !e_idx || !t_in || !t_out) {
        set_error("ts_search_brute_noalloc: NULL output array");
        return TS_ERR_INVALID_ARG;
    }
    k_na_tiles<1><<<grid, NA_WARPS * 32, 0, s>>>(P);
    TS_LAUNCHED();
    TS_CUDA(cudaMemcpyAsync(&h, scratch, sizeof(NaCtrl), cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaStreamSynchronize(s));
    return na_status(h.status);
}

}  // namespace ts
