// ts_prims.cu -- device primitives: exclusive scans and a stable LSD radix sort.
//
// Index building sorts segment keys and turns bin counts into offset arrays (radix sort plus
// prefix sums, the GB300 form of the paper's sorted arrays and bin ranges, Sec. 4.1-4.3); the
// search scans per-tile hit counts into output offsets. All of it is hand-written here.
#include <stdarg.h>
#include <stdio.h>

#include <atomic>

#include <algorithm>
#include <mutex>

#include "ts_internal.cuh"

namespace ts {

// ---------------------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------------------
static thread_local char g_err[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

const char *last_error() { return g_err; }

ts_status cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) {
        set_error("out of device memory in %s", what);
        cudaGetLastError();
        return TS_ERR_OOM;
    }
    set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
    return TS_ERR_CUDA;
}

void DevBuf::release()
{
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
}

// The library's stream-ordered pool of a device: freed blocks stay in the pool (no release
// threshold), so the work buffers of repeated searches are not mapped and unmapped every call.
static cudaMemPool_t work_pool()
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = pool;
    }
    return pools[dev];
}

void pool_trim()
{
    cudaMemPool_t pool = work_pool();
    if (pool && cudaDeviceSynchronize() == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    cudaGetLastError();
}

cudaError_t pool_malloc(void **p, size_t nbytes, cudaStream_t stream)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(stream, &cs);
    cudaMemPool_t pool = cs == cudaStreamCaptureStatusNone ? work_pool() : nullptr;
    return pool ? cudaMallocFromPoolAsync(p, nbytes, pool, stream)
                : cudaMallocAsync(p, nbytes, stream);
}

ts_status DevBuf::alloc(size_t nbytes, cudaStream_t stream)
{
    release();
    s = stream;
    bytes = nbytes;
    if (nbytes == 0) nbytes = 256;
    cudaError_t e = pool_malloc(&p, nbytes, stream);
    if (e != cudaSuccess) {
        p = nullptr;
        return cuda_status(e, "cudaMallocAsync");
    }
    return TS_OK;
}

// ---------------------------------------------------------------------------------------------
// scan
// ---------------------------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ inline T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive prefix, *total the sum.
template <class T>
__device__ inline T block_excl_scan(T v, T *total)
{
    __shared__ T warp_sums[SCAN_THREADS / 32 + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        T w = lane < SCAN_THREADS / 32 ? warp_sums[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = wi - w;
        if (lane == SCAN_THREADS / 32 - 1) warp_sums[SCAN_THREADS / 32] = wi;  // total
    }
    __syncthreads();
    T excl = warp_sums[wid] + incl - v;
    if (total) *total = warp_sums[SCAN_THREADS / 32];
    __syncthreads();
    return excl;
}

// Element count of a primitive: the capacity, or the smaller count held in device memory (a
// run whose size is known only on the device, e.g. a replayed CUDA graph).
__device__ __forceinline__ uint64_t dev_count(uint64_t cap, const uint32_t *n_dev)
{
    return n_dev ? min(cap, (uint64_t)*n_dev) : cap;
}

template <class Tin, class Tout>
__global__ void k_tile_sums(const Tin *in, uint64_t ncap, const uint32_t *n_dev, Tout *sums)
{
    pdl_enter();
    const uint64_t n = dev_count(ncap, n_dev);
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    if (base >= n) {
        if (threadIdx.x == 0) sums[blockIdx.x] = 0;
        return;
    }
    Tout acc = 0;
    for (int k = 0; k < SCAN_ITEMS; k++) {
        uint64_t i = base + (uint64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) acc += (Tout)in[i];
    }
    Tout total;
    block_excl_scan<Tout>(acc, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Scan one tile per block with the tile's starting offset taken from `tile_off` (or 0), writing
// out[i] = exclusive prefix; the block whose tile holds index n writes out[n] = total.
template <class Tin, class Tout>
__global__ void k_tile_scan(const Tin *in, uint64_t ncap, const uint32_t *n_dev,
                            const Tout *tile_off, Tout *out)
{
    pdl_enter();
    const uint64_t n = dev_count(ncap, n_dev);
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    if (base > n) return;
    Tout v[SCAN_ITEMS];
    Tout acc = 0;
    // thread-contiguous items for a stable sequential order within a thread
    uint64_t tbase = base + (uint64_t)threadIdx.x * SCAN_ITEMS;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        uint64_t i = tbase + k;
        v[k] = i < n ? (Tout)in[i] : Tout(0);
        acc += v[k];
    }
    Tout total;
    Tout pre = block_excl_scan<Tout>(acc, &total);
    Tout off = (tile_off ? tile_off[blockIdx.x] : Tout(0)) + pre;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        uint64_t i = tbase + k;
        if (i < n) out[i] = off;
        off += v[k];
    }
    if (threadIdx.x == 0 && n < base + SCAN_TILE)
        out[n] = (tile_off ? tile_off[blockIdx.x] : Tout(0)) + total;
}

// Second pass of a two-kernel scan: every block first adds up the totals of the tiles before its
// own (at most SCAN_LOOKBACK of them, read by the whole block), then scans its tile.
constexpr uint64_t SCAN_LOOKBACK = 4096;

template <class Tin, class Tout>
__global__ void k_tile_scan_lb(const Tin *in, uint64_t ncap, const uint32_t *n_dev,
                               const Tout *sums, Tout *out)
{
    pdl_enter();
    const uint64_t n = dev_count(ncap, n_dev);
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    if (base > n) return;
    Tout pre = 0;
    for (uint32_t j = threadIdx.x; j < blockIdx.x; j += SCAN_THREADS) pre += sums[j];
    Tout before;
    block_excl_scan<Tout>(pre, &before);
    Tout v[SCAN_ITEMS];
    Tout acc = 0;
    const uint64_t tbase = base + (uint64_t)threadIdx.x * SCAN_ITEMS;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        const uint64_t i = tbase + k;
        v[k] = i < n ? (Tout)in[i] : Tout(0);
        acc += v[k];
    }
    Tout total;
    Tout off = before + block_excl_scan<Tout>(acc, &total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        const uint64_t i = tbase + k;
        if (i < n) out[i] = off;
        off += v[k];
    }
    if (threadIdx.x == 0 && n < base + SCAN_TILE) out[n] = before + total;
}

// Exclusive scan of n (or *n_dev <= n) values: out[0..n] with out[n] = total. One block per tile
// of SCAN_TILE values plus one, so that the tile holding index n always exists.
template <class Tin, class Tout>
static ts_status scan_impl(const Tin *in, Tout *out, uint64_t n, const uint32_t *n_dev,
                           cudaStream_t s)
{
    if (n == 0) {
        TS_CUDA(cudaMemsetAsync(out, 0, sizeof(Tout), s));
        return TS_OK;
    }
    const uint64_t nt = n / SCAN_TILE + 1;
    if (nt == 1) {
        TS_LAUNCH_PDL(k_tile_scan<Tin, Tout>, dim3(1), dim3(SCAN_THREADS), 0, s,
                      in, n, n_dev, nullptr, out);
        return TS_OK;
    }
    DevBuf sums;
    TS_CHECK(sums.alloc(sizeof(Tout) * nt, s));
    TS_LAUNCH_PDL(k_tile_sums<Tin, Tout>, dim3((unsigned)nt), dim3(SCAN_THREADS), 0, s,
                  in, n, n_dev, sums.as<Tout>());
    if (nt <= SCAN_LOOKBACK) {
        TS_LAUNCH_PDL(k_tile_scan_lb<Tin, Tout>, dim3((unsigned)nt), dim3(SCAN_THREADS), 0, s,
                      in, n, n_dev, sums.as<Tout>(), out);
        return TS_OK;
    }
    DevBuf offs;
    TS_CHECK(offs.alloc(sizeof(Tout) * (nt + 1), s));
    TS_CHECK((scan_impl<Tout, Tout>(sums.as<Tout>(), offs.as<Tout>(), nt, nullptr, s)));
    TS_LAUNCH_PDL(k_tile_scan<Tin, Tout>, dim3((unsigned)nt), dim3(SCAN_THREADS), 0, s,
                  in, n, n_dev, offs.as<Tout>(), out);
    return TS_OK;
}

ts_status scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t n, cudaStream_t s,
                          const uint32_t *n_dev)
{
    return scan_impl<uint32_t, uint64_t>(in, out, n, n_dev, s);
}

__global__ void k_narrow_u64(const uint64_t *in, uint32_t *out, uint64_t ncap,
                             const uint32_t *n_dev, uint32_t *status)
{
    pdl_enter();
    const uint64_t n = dev_count(ncap, n_dev);
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    uint64_t v = in[i];
    if (v > 0xffffffffull) {
        atomicOr(status, DEV_ERR_OVERFLOW);
        v = 0xffffffffull;
    }
    out[i] = (uint32_t)v;
}

ts_status scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *status,
                   cudaStream_t s, const uint32_t *n_dev)
{
    DevBuf wide;
    TS_CHECK(wide.alloc(sizeof(uint64_t) * (n + 1), s));
    TS_CHECK(scan_u32_to_u64(in, wide.as<uint64_t>(), n, s, n_dev));
    TS_LAUNCH_PDL(k_narrow_u64, dim3((unsigned)((n + 1 + 255) / 256)), dim3(256), 0, s,
                  wide.as<uint64_t>(), out, n, n_dev, status);
    return TS_OK;
}

// ---------------------------------------------------------------------------------------------
// radix sort: LSD, 8-bit digits, 256 threads x 8 keys per block tile. Each pass: per-tile digit
// histograms (digit-major), an exclusive scan of them, and a stable scatter in which every warp
// ranks its 256 consecutive keys with __match_any_sync and the block adds the earlier warps'
// counts.
// ---------------------------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_RADIX = 256;

template <class K>
__global__ void k_rs_hist(const K *keys, uint64_t ncap, const uint32_t *n_dev, int shift,
                          uint32_t *hist, uint32_t ntiles)
{
    pdl_enter();
    __shared__ uint32_t h[RS_RADIX];
    const uint64_t n = dev_count(ncap, n_dev);
    for (int i = threadIdx.x; i < RS_RADIX; i += RS_THREADS) h[i] = 0;
    __syncthreads();
    uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
    for (int k = 0; k < RS_ITEMS; k++) {
        uint64_t i = base + (uint64_t)k * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    for (int dgt = threadIdx.x; dgt < RS_RADIX; dgt += RS_THREADS)
        hist[(uint64_t)dgt * ntiles + blockIdx.x] = h[dgt];
}

template <class K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const K *keys_in, const uint32_t *vals_in,
                                                           K *keys_out, uint32_t *vals_out,
                                                           uint64_t ncap, const uint32_t *n_dev,
                                                           int shift, const uint64_t *digit_off,
                                                           uint32_t ntiles)
{
    pdl_enter();
    __shared__ uint32_t wcnt[RS_WARPS][RS_RADIX];
    const uint64_t n = dev_count(ncap, n_dev);
    if ((uint64_t)blockIdx.x * RS_TILE >= n) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_RADIX; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint64_t wbase = (uint64_t)blockIdx.x * RS_TILE + (uint64_t)wid * (RS_ITEMS * 32);
    K key[RS_ITEMS];
    uint32_t val[RS_ITEMS];
    uint32_t rank[RS_ITEMS];
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < RS_ITEMS; k++) {
        uint64_t i = wbase + (uint64_t)k * 32 + lane;
        bool ok = i < n;
        key[k] = ok ? keys_in[i] : K(0);
        val[k] = ok ? vals_in[i] : 0u;
        uint32_t dgt = ok ? ((uint32_t)(key[k] >> shift) & 0xffu) : 0x100u;
        uint32_t peers = __match_any_sync(0xffffffffu, dgt);
        uint32_t before = __popc(peers & lt_mask);
        uint32_t leader = __ffs(peers) - 1;
        uint32_t cur = 0;
        if (ok && lane == (int)leader) {
            cur = wcnt[wid][dgt];
            wcnt[wid][dgt] = cur + __popc(peers);
        }
        cur = __shfl_sync(0xffffffffu, cur, leader);
        rank[k] = cur + before;
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps, per digit
    for (int dgt = threadIdx.x; dgt < RS_RADIX; dgt += RS_THREADS) {
        uint32_t run = 0;
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t c = wcnt[w][dgt];
            wcnt[w][dgt] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RS_ITEMS; k++) {
        uint64_t i = wbase + (uint64_t)k * 32 + lane;
        if (i >= n) continue;
        uint32_t dgt = (uint32_t)(key[k] >> shift) & 0xffu;
        uint64_t dst = digit_off[(uint64_t)dgt * ntiles + blockIdx.x] + wcnt[wid][dgt] + rank[k];
        keys_out[dst] = key[k];
        vals_out[dst] = val[k];
    }
}

// Scatter of one pass that computes its own digit offsets from the per-tile histograms (for at
// most RS_FUSED_TILES tiles): thread d adds up digit d over all tiles and over the tiles before
// this block's, and a block scan over the digit totals gives every digit's first position.
constexpr uint32_t RS_FUSED_TILES = 256;

template <class K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter_fused(const K *keys_in,
                                                                 const uint32_t *vals_in,
                                                                 K *keys_out, uint32_t *vals_out,
                                                                 uint64_t ncap, const uint32_t *n_dev,
                                                                 int shift, const uint32_t *hist,
                                                                 uint32_t ntiles)
{
    pdl_enter();
    __shared__ uint32_t wcnt[RS_WARPS][RS_RADIX];
    __shared__ uint32_t dbase[RS_RADIX];
    const uint64_t n = dev_count(ncap, n_dev);
    if ((uint64_t)blockIdx.x * RS_TILE >= n) return;
    {
        const int d = threadIdx.x;  // RS_THREADS == RS_RADIX
        uint32_t tot = 0, pre = 0;
        for (uint32_t t = 0; t < ntiles; t++) {
            const uint32_t v = hist[(uint64_t)d * ntiles + t];
            tot += v;
            pre += t < blockIdx.x ? v : 0u;
        }
        uint32_t all;
        const uint32_t base = block_excl_scan<uint32_t>(tot, &all);
        dbase[d] = base + pre;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_RADIX; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint64_t wbase = (uint64_t)blockIdx.x * RS_TILE + (uint64_t)wid * (RS_ITEMS * 32);
    K key[RS_ITEMS];
    uint32_t val[RS_ITEMS];
    uint32_t rank[RS_ITEMS];
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < RS_ITEMS; k++) {
        uint64_t i = wbase + (uint64_t)k * 32 + lane;
        bool ok = i < n;
        key[k] = ok ? keys_in[i] : K(0);
        val[k] = ok ? vals_in[i] : 0u;
        uint32_t dgt = ok ? ((uint32_t)(key[k] >> shift) & 0xffu) : 0x100u;
        uint32_t peers = __match_any_sync(0xffffffffu, dgt);
        uint32_t before = __popc(peers & lt_mask);
        uint32_t leader = __ffs(peers) - 1;
        uint32_t cur = 0;
        if (ok && lane == (int)leader) {
            cur = wcnt[wid][dgt];
            wcnt[wid][dgt] = cur + __popc(peers);
        }
        cur = __shfl_sync(0xffffffffu, cur, leader);
        rank[k] = cur + before;
        __syncwarp();
    }
    __syncthreads();
    for (int dgt = threadIdx.x; dgt < RS_RADIX; dgt += RS_THREADS) {
        uint32_t run = 0;
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t c = wcnt[w][dgt];
            wcnt[w][dgt] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RS_ITEMS; k++) {
        uint64_t i = wbase + (uint64_t)k * 32 + lane;
        if (i >= n) continue;
        uint32_t dgt = (uint32_t)(key[k] >> shift) & 0xffu;
        uint64_t dst = (uint64_t)dbase[dgt] + wcnt[wid][dgt] + rank[k];
        keys_out[dst] = key[k];
        vals_out[dst] = val[k];
    }
}

template <class K>
__global__ void k_copy_kv(const K *ks, const uint32_t *vs, K *kd, uint32_t *vd, uint64_t ncap,
                          const uint32_t *n_dev)
{
    pdl_enter();
    const uint64_t n = dev_count(ncap, n_dev);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        kd[i] = ks[i];
        vd[i] = vs[i];
    }
}

template <class K>
static ts_status radix_sort_impl(K *keys, uint32_t *vals, uint64_t n, int bits, cudaStream_t s,
                                 const uint32_t *n_dev)
{
    if (n <= 1 || bits <= 0) return TS_OK;
    uint32_t ntiles = (uint32_t)((n + RS_TILE - 1) / RS_TILE);
    DevBuf kb, vb, hist, off;
    TS_CHECK(kb.alloc(sizeof(K) * n, s));
    TS_CHECK(vb.alloc(sizeof(uint32_t) * n, s));
    uint64_t nh = (uint64_t)RS_RADIX * ntiles;
    TS_CHECK(hist.alloc(sizeof(uint32_t) * nh, s));
    const bool fused = ntiles <= RS_FUSED_TILES && n < (1ull << 32);
    if (!fused) TS_CHECK(off.alloc(sizeof(uint64_t) * (nh + 1), s));
    K *ka = keys, *kbp = kb.as<K>();
    uint32_t *va = vals, *vbp = vb.as<uint32_t>();
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        TS_LAUNCH_PDL(k_rs_hist<K>, dim3(ntiles), dim3(RS_THREADS), 0, s, ka, n, n_dev, shift,
                      hist.as<uint32_t>(), ntiles);
        if (fused) {
            TS_LAUNCH_PDL(k_rs_scatter_fused<K>, dim3(ntiles), dim3(RS_THREADS), 0, s, ka, va, kbp,
                          vbp, n, n_dev, shift, hist.as<uint32_t>(), ntiles);
        } else {
            TS_CHECK(scan_u32_to_u64(hist.as<uint32_t>(), off.as<uint64_t>(), nh, s));
            TS_LAUNCH_PDL(k_rs_scatter<K>, dim3(ntiles), dim3(RS_THREADS), 0, s, ka, va, kbp, vbp,
                          n, n_dev, shift, off.as<uint64_t>(), ntiles);
        }
        K *tk = ka; ka = kbp; kbp = tk;
        uint32_t *tv = va; va = vbp; vbp = tv;
    }
    if (ka != keys) {
        if (n_dev) {
            const unsigned cb = (unsigned)std::min<uint64_t>((n + 255) / 256, 152 * 8);
            TS_LAUNCH_PDL(k_copy_kv<K>, dim3(cb), dim3(256), 0, s, ka, va, keys, vals, n, n_dev);
        } else {
            TS_CUDA(cudaMemcpyAsync(keys, ka, sizeof(K) * n, cudaMemcpyDeviceToDevice, s));
            TS_CUDA(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
        }
    }
    return TS_OK;
}

ts_status radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t n, int bits, cudaStream_t s,
                         const uint32_t *n_dev)
{
    return radix_sort_impl<uint64_t>(keys, vals, n, bits, s, n_dev);
}

ts_status radix_sort_u32(uint32_t *keys, uint32_t *vals, uint64_t n, int bits, cudaStream_t s,
                         const uint32_t *n_dev)
{
    return radix_sort_impl<uint32_t>(keys, vals, n, bits, s, n_dev);
}

}  // namespace ts
