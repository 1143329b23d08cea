// ts_internal.cuh -- shared declarations of the GB300 trajectory search library.
//
// Data layout in HBM (all arrays 256-byte aligned by cudaMalloc):
//   SegD  : 64 B per entry, FP64 start point, start time, velocity, end time (exact test)
//   RecF  : 32 B per entry, FP32 MBB rounded outward + start/end time rounded outward
//           (conservative prefilter)
//   Entries are stored in start-time order (Sec. 4.2); the spatiotemporal id arrays (Sec. 4.3)
//   and the grid lookup array (Sec. 4.1) keep a duplicated RecF next to every id so candidate
//   ranges stream contiguously.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <utility>

#include "../../include/ts.h"

namespace ts {

// ---------------------------------------------------------------------------------------------
// records
// ---------------------------------------------------------------------------------------------
struct __align__(16) RecF {
    float xmin, xmax;  // each axis as an adjacent (min, max) pair: one 8-byte load per axis
    float ymin, ymax;
    float zmin, zmax;
    float t0, t1;      // t0 rounded toward -inf, t1 toward +inf
};
static_assert(sizeof(RecF) == 32, "RecF is 32 bytes");

struct __align__(16) SegD {
    double x0, y0, z0, t0;
    double vx, vy, vz, t1;
};
static_assert(sizeof(SegD) == 64, "SegD is 64 bytes");

// Exact data of one query segment: its position at the start w0 of its clipped window [w0, w1],
// its velocity, and minus the request's d^2 (the addend of c, stored negated so that no FP64
// instruction negates it).
struct __align__(16) QueryD {
    double xw, yw, zw, w0;
    double vx, vy, vz, w1;
    double ndd, pad;
};
static_assert(sizeof(QueryD) == 80, "QueryD is 80 bytes");

// Query group: up to 32 consecutive (sorted) queries sharing one candidate array and range.
struct Group {
    uint32_t first;  // first sorted query
    uint32_t count;  // 1..32
    uint32_t sel;    // 0,1,2: X/Y/Z id array; 3: time-sorted entries; 4: grid lookup array
    uint32_t lo, hi; // union of the members' candidate ranges [lo, hi)
    uint32_t pad[3];
};

enum : uint32_t { SEL_X = 0, SEL_Y = 1, SEL_Z = 2, SEL_T = 3, SEL_GRID = 4 };

// Status bits written by kernels (device status word).
enum : uint32_t {
    DEV_ERR_INVALID = 1u,   // NaN/Inf or t1 <= t0 in an input segment
    DEV_ERR_TIMEOUT = 2u,   // a bounded wait ran out
    DEV_ERR_INTERNAL = 4u,  // an internal consistency check failed
    DEV_ERR_OVERFLOW = 8u   // a 32-bit offset would overflow
};

// Stats slots (u64 array in device memory).
enum : int {
    ST_QSEGS = 0, ST_TESTS = 1, ST_EXACT = 2, ST_HITS = 3, ST_TILES = 4, ST_GROUPS = 5,
    ST_SUBBIN = 6, ST_SCRATCH = 7,  // ST_SCRATCH: hits offered to the scratch
    // pair kernel sweep (count pass): chunks swept, chunks swept by the two-axis bitmask, member
    // visits of the sparse path, survivors of the bitmask given the full FP32 filters
    ST_CHUNKS = 8, ST_DENSE = 9, ST_SPARSE = 10, ST_STAGE2 = 11, ST_NSLOTS = 12
};

// ---------------------------------------------------------------------------------------------
// order-preserving integer keys of doubles (finite values; -0.0 canonicalised to +0.0)
// ---------------------------------------------------------------------------------------------
__host__ __device__ inline uint64_t dkey(double x)
{
    x = x + 0.0;  // -0.0 -> +0.0
#ifdef __CUDA_ARCH__
    uint64_t u = (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    memcpy(&u, &x, 8);
#endif
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

__host__ __device__ inline double dkey_inv(uint64_t k)
{
    uint64_t u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, 8);
    return x;
#endif
}

// ---------------------------------------------------------------------------------------------
// 1-D uniform partition (subbins of Sec. 4.3, grid cells of Sec. 4.1): part j is
// [lo + j*w, lo + (j+1)*w), the last part unbounded above. part_of(x) = largest j in [0, v-1]
// with lo + j*w <= x, or -1 when x < lo. The boundaries are evaluated exactly as written
// (library compiled without FMA contraction) so the part of a value never depends on rounding
// of a division.
// ---------------------------------------------------------------------------------------------
__host__ __device__ inline double part_bound(double lo, double w, int j)
{
    return lo + (double)j * w;
}

__host__ __device__ inline int part_of(double x, double lo, double w, int v)
{
    if (!(x >= lo)) return -1;
    if (v <= 1 || !(w > 0.0)) return v - 1;
    double f = floor((x - lo) / w);
    int j;
    if (!(f < (double)v)) j = v - 1;
    else if (f < 0.0) j = 0;
    else j = (int)f;
    while (j + 1 < v && part_bound(lo, w, j + 1) <= x) j++;
    while (j > 0 && part_bound(lo, w, j) > x) j--;
    return j;
}


// ---------------------------------------------------------------------------------------------
// host-side error plumbing
// ---------------------------------------------------------------------------------------------
void set_error(const char *fmt, ...);
ts_status cuda_status(cudaError_t e, const char *what);

#define TS_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e__ = (call);                                                      \
        if (e__ != cudaSuccess) return ::ts::cuda_status(e__, #call);                  \
    } while (0)

// Count one kernel launch of this library and surface launch errors.
void note_launch();
#define TS_LAUNCHED()                                                                  \
    do {                                                                               \
        ::ts::note_launch();                                                           \
        TS_CUDA(cudaGetLastError());                                                   \
    } while (0)

// Programmatic dependent launch: a kernel launched with launch_pdl may be scheduled while its
// predecessor on the stream is still running. Every such kernel starts with pdl_enter(): it
// waits there until the predecessor grid has completed and its memory is visible (so it reads
// nothing early), then lets its own successor be scheduled (which happens only once every block
// of this grid has started, so early successors never hold the SMs this grid still needs).
// Launched without the attribute, pdl_enter() returns at once.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

#define TS_LAUNCH_PDL(...)                                                             \
    do {                                                                               \
        ::ts::note_launch();                                                           \
        TS_CUDA(::ts::launch_pdl(__VA_ARGS__));                                        \
    } while (0)

#define TS_CHECK(st)                                                                   \
    do {                                                                               \
        ts_status s__ = (st);                                                          \
        if (s__ != TS_OK) return s__;                                                  \
    } while (0)

// Stream-ordered device buffer (cudaMallocAsync / cudaFreeAsync).
// Stream-ordered allocation from the library's pool (freed blocks stay pooled); inside a stream
// capture a graph memory node. Release with cudaFreeAsync.
cudaError_t pool_malloc(void **p, size_t nbytes, cudaStream_t stream);
// Return the pool's unused memory of the current device to the device (synchronises it).
void pool_trim();

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes), s(o.s) { o.p = nullptr; o.bytes = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept
    {
        if (this != &o) {
            release();
            p = o.p; bytes = o.bytes; s = o.s;
            o.p = nullptr; o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void release();
    ts_status alloc(size_t nbytes, cudaStream_t stream);
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// ---------------------------------------------------------------------------------------------
// primitives (ts_prims.cu)
// ---------------------------------------------------------------------------------------------
// The primitives take a capacity n and optionally n_dev, a device word holding the actual count
// (<= n) of a run whose size only the device knows; the work then follows the actual count.
// exclusive scan of n u32 values into n+1 u64 offsets (out[n] = total)
ts_status scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t n, cudaStream_t s,
                          const uint32_t *n_dev = nullptr);
// exclusive scan of n u32 values into n+1 u32 offsets; sets DEV_ERR_OVERFLOW in *status when the
// total does not fit in 32 bits
ts_status scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *status,
                   cudaStream_t s, const uint32_t *n_dev = nullptr);
// stable LSD radix sort of (key, value) pairs by the low `bits` bits of the key
ts_status radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t n, int bits, cudaStream_t s,
                         const uint32_t *n_dev = nullptr);
ts_status radix_sort_u32(uint32_t *keys, uint32_t *vals, uint64_t n, int bits, cudaStream_t s,
                         const uint32_t *n_dev = nullptr);

}  // namespace ts

// Library-internal entry points shared between translation units.
namespace ts {
struct Index;
struct SearchOut;
ts_status build_index(const ts_segments *db, const ts_index_params *p, cudaStream_t s,
                      Index **out);
void destroy_index(Index *idx);
}  // namespace ts
