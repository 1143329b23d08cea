// ts_index.cu -- building the resident index on the device.
//
// Steps (all device kernels; the host only picks parameters from exact reductions):
//   ingest   : validate (finite, t1 > t0), order keys of t_start, exact extents   (Sec. 3.1)
//   sort     : stable radix sort by t_start, ties by input index                     (Sec. 4.2)
//   gather   : FP64 exact records (velocity precomputed) and FP32 outward-rounded
//              prefilter records in sorted order
//   bins     : m temporal bins, B_j^start, B_j^end, first/last offsets, prefix max   (Sec. 4.2)
//   subbins  : per dimension, (subbin, entry) keys -> radix sort -> X/Y/Z id arrays and
//              (subbin, bin) offsets                                                 (Sec. 4.3)
//   grid     : per entry its MBB's cells -> (cell, entry) keys -> radix sort -> lookup array A
//              and dense cell offsets                                                (Sec. 4.1)
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ts_index.cuh"

namespace ts {

namespace {

constexpr int TPB = 256;

inline unsigned nblocks(uint64_t n, int tpb = TPB)
{
    uint64_t b = (n + tpb - 1) / tpb;
    return (unsigned)(b ? b : 1);
}

// reduction slots (order keys): 0 min t0, 1 max t1, 2 max duration, 3..5 min emin, 6..8 max
// emax, 9..11 max extent
enum { R_TMIN = 0, R_TMAX = 1, R_DUR = 2, R_EMIN = 3, R_EMAX = 6, R_LONG = 9, R_N = 12 };

__device__ inline bool finite_d(double x) { return isfinite(x); }

__device__ inline unsigned long long warp_min_u64(unsigned long long v)
{
    for (int o = 16; o; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

__device__ inline unsigned long long warp_max_u64(unsigned long long v)
{
    for (int o = 16; o; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

struct SegIn {
    const double *f[8];
};

__global__ void k_init_red(unsigned long long *red)
{
    int i = threadIdx.x;
    if (i >= R_N) return;
    bool is_min = (i == R_TMIN) || (i >= R_EMIN && i < R_EMIN + 3);
    red[i] = is_min ? ~0ull : 0ull;
}

__global__ void k_ingest(SegIn in, uint64_t n, uint64_t *keys, uint32_t *vals,
                         unsigned long long *red, uint32_t *status)
{
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = i < n;
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = ok ? in.f[k][i] : 0.0;
    bool valid = true;
#pragma unroll
    for (int k = 0; k < 8; k++) valid = valid && finite_d(v[k]);
    valid = valid && (v[7] > v[3]);
    if (ok && !valid) atomicOr(status, DEV_ERR_INVALID);
    if (ok) {
        keys[i] = dkey(v[3]);
        vals[i] = (uint32_t)i;
    }
    bool use = ok && valid;
    unsigned long long r[R_N];
    r[R_TMIN] = use ? dkey(v[3]) : ~0ull;
    r[R_TMAX] = use ? dkey(v[7]) : 0ull;
    r[R_DUR] = use ? dkey(v[7] - v[3]) : 0ull;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        double lo = v[d] < v[4 + d] ? v[d] : v[4 + d];
        double hi = v[d] < v[4 + d] ? v[4 + d] : v[d];
        r[R_EMIN + d] = use ? dkey(lo) : ~0ull;
        r[R_EMAX + d] = use ? dkey(hi) : 0ull;
        r[R_LONG + d] = use ? dkey(hi - lo) : 0ull;
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < R_N; k++) {
        bool is_min = (k == R_TMIN) || (k >= R_EMIN && k < R_EMIN + 3);
        unsigned long long w = is_min ? warp_min_u64(r[k]) : warp_max_u64(r[k]);
        if (lane == 0) {
            if (is_min) atomicMin(&red[k], w);
            else atomicMax(&red[k], w);
        }
    }
}

// Outward rounding of an FP64 interval to FP32 (conservative prefilter boxes).
__device__ inline float f_dn(double x) { return __double2float_rd(x); }
__device__ inline float f_up(double x) { return __double2float_ru(x); }

__global__ void k_gather(SegIn in, uint64_t n, const uint32_t *perm, SegD *seg, RecF *rec,
                         uint32_t *orig)
{
    uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint32_t i = perm[s];
    double x0 = in.f[0][i], y0 = in.f[1][i], z0 = in.f[2][i], t0 = in.f[3][i];
    double x1 = in.f[4][i], y1 = in.f[5][i], z1 = in.f[6][i], t1 = in.f[7][i];
    double dt = t1 - t0;
    SegD d;
    d.x0 = x0; d.y0 = y0; d.z0 = z0; d.t0 = t0; d.t1 = t1;
    d.vx = (x1 - x0) / dt;
    d.vy = (y1 - y0) / dt;
    d.vz = (z1 - z0) / dt;
    seg[s] = d;
    RecF r;
    r.xmin = f_dn(fmin(x0, x1)); r.xmax = f_up(fmax(x0, x1));
    r.ymin = f_dn(fmin(y0, y1)); r.ymax = f_up(fmax(y0, y1));
    r.zmin = f_dn(fmin(z0, z1)); r.zmax = f_up(fmax(z0, z1));
    r.t0 = f_dn(t0); r.t1 = f_up(t1);
    rec[s] = r;
    orig[s] = i;
}

// Key of an entry inside its bin: (bin, x of its FP32 box centre as an order-preserving integer).
// Any order inside a bin leaves every bin's range unchanged; x order makes aligned chunks of 64
// entries narrow in x, so a chunk's bounding record rejects most queries.
__global__ void k_tx_key(const RecF *rec, const uint32_t *bin_of, uint64_t n, uint64_t *keys,
                         uint32_t *vals)
{
    const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const RecF r = rec[s];
    uint32_t u = __float_as_uint(0.5f * r.xmin + 0.5f * r.xmax + 0.0f);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    keys[s] = ((uint64_t)bin_of[s] << 32) | u;
    vals[s] = (uint32_t)s;
}

// Bounding record of every aligned chunk of 64 records, a warp per chunk.
__global__ void k_chunk_box(const RecF *rec, uint64_t n, uint64_t nchunks, RecF *box)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t c = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks;
         c += warps) {
        float lo[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
        float hi[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
        for (int h = 0; h < 2; h++) {
            const uint64_t i = c * 64 + h * 32 + lane;
            if (i < n) {
                const RecF r = rec[i];
                lo[0] = fminf(lo[0], r.xmin); hi[0] = fmaxf(hi[0], r.xmax);
                lo[1] = fminf(lo[1], r.ymin); hi[1] = fmaxf(hi[1], r.ymax);
                lo[2] = fminf(lo[2], r.zmin); hi[2] = fmaxf(hi[2], r.zmax);
                lo[3] = fminf(lo[3], r.t0); hi[3] = fmaxf(hi[3], r.t1);
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
#pragma unroll
            for (int k = 0; k < 4; k++) {
                lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
                hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
            }
        if (lane == 0) {
            RecF b;
            b.xmin = lo[0]; b.xmax = hi[0];
            b.ymin = lo[1]; b.ymax = hi[1];
            b.zmin = lo[2]; b.zmax = hi[2];
            b.t0 = lo[3]; b.t1 = hi[3];
            box[c] = b;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// temporal bins
// ---------------------------------------------------------------------------------------------
__global__ void k_bins_init(uint32_t m, double tmin, double b, double *bin_start,
                            unsigned long long *end_key)
{
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    bin_start[j] = part_bound(tmin, b, (int)j);
    end_key[j] = dkey(part_bound(tmin, b, (int)j + 1));
}

__global__ void k_bin_of(const SegD *seg, uint64_t n, uint32_t m, double tmin, double b,
                         uint32_t *bin_of, unsigned long long *end_key)
{
    uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int j = part_of(seg[s].t0, tmin, b, (int)m);
    if (j < 0) j = 0;  // t0 >= tmin always
    bin_of[s] = (uint32_t)j;
    atomicMax(&end_key[j], dkey(seg[s].t1));
}

// off[j] = first sorted entry with bin >= j (bin_of is non-decreasing)
__global__ void k_bin_bounds(const uint32_t *bin_of, uint64_t n, uint32_t m, uint32_t *off)
{
    uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint32_t j = bin_of[s];
    uint32_t jp = s ? bin_of[s - 1] + 1 : 0;
    for (uint32_t k = jp; k <= j; k++) off[k] = (uint32_t)s;
    if (s == n - 1)
        for (uint32_t k = j + 1; k <= m; k++) off[k] = (uint32_t)n;
}

__global__ void k_bin_end_final(const unsigned long long *end_key, uint32_t m, double *bin_end)
{
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) bin_end[j] = dkey_inv(end_key[j]);
}

// prefix maximum over the bins (one block)
__global__ void k_prefix_max(const double *in, uint32_t m, double *out)
{
    __shared__ double tot[1024];
    uint32_t per = (m + blockDim.x - 1) / blockDim.x;
    uint32_t a = threadIdx.x * per, bnd = min(m, a + per);
    double run = -INFINITY;
    for (uint32_t j = a; j < bnd; j++) run = fmax(run, in[j]);
    tot[threadIdx.x] = run;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = -INFINITY;
        for (unsigned t = 0; t < blockDim.x; t++) {
            double v = tot[t];
            tot[t] = r;
            r = fmax(r, v);
        }
    }
    __syncthreads();
    run = tot[threadIdx.x];
    for (uint32_t j = a; j < bnd; j++) {
        run = fmax(run, in[j]);
        out[j] = run;
    }
}

// ---------------------------------------------------------------------------------------------
// partitions (subbins / grid)
// ---------------------------------------------------------------------------------------------
// Per-dimension MBB of a sorted entry, taken from the caller's original endpoints (exact).
__global__ void k_mbb(SegIn in, const uint32_t *orig, uint64_t n, int dim, double *lo, double *hi)
{
    uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint32_t i = orig[s];
    double a = in.f[dim][i], b = in.f[4 + dim][i];
    lo[s] = a < b ? a : b;
    hi[s] = a < b ? b : a;
}

__global__ void k_part_count(const double *lo, const double *hi, uint64_t n, double plo, double pw,
                             int v, uint32_t *cnt)
{
    uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int a = part_of(lo[s], plo, pw, v);
    int b = part_of(hi[s], plo, pw, v);
    if (a < 0) a = 0;
    cnt[s] = b >= a ? (uint32_t)(b - a + 1) : 0u;
}

__global__ void k_part_emit(const double *lo, const double *hi, uint64_t n, double plo, double pw,
                            int v, const uint32_t *pos, uint32_t *keys, uint32_t *vals)
{
    uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int a = part_of(lo[s], plo, pw, v);
    int b = part_of(hi[s], plo, pw, v);
    if (a < 0) a = 0;
    uint32_t p = pos[s];
    for (int j = a; j <= b; j++, p++) {
        keys[p] = (uint32_t)j;
        vals[p] = (uint32_t)s;
    }
}

__global__ void k_st_hist(const uint32_t *keys, const uint32_t *ids, uint64_t len,
                          const uint32_t *bin_of, uint32_t m, uint32_t *cnt)
{
    uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= len) return;
    atomicAdd(&cnt[(uint64_t)keys[p] * m + bin_of[ids[p]]], 1u);
}

__global__ void k_gather_rec(const uint32_t *ids, uint64_t len, const RecF *rec, RecF *out)
{
    uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < len) out[p] = rec[ids[p]];
}

// grid: every sorted entry is keyed by the cell of its MBB's minimum corner (single assignment)
__global__ void k_grid_key(const double *lo3, uint64_t n, double gx, double gy, double gz,
                           double wx, double wy, double wz, int g, uint32_t *keys, uint32_t *vals)
{
    uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double plo[3] = {gx, gy, gz}, pw[3] = {wx, wy, wz};
    uint32_t c[3];
    for (int d = 0; d < 3; d++) {
        int a = part_of(lo3[(uint64_t)d * n + s], plo[d], pw[d], g);
        c[d] = (uint32_t)(a < 0 ? 0 : a);
    }
    keys[s] = (c[0] * (uint32_t)g + c[1]) * (uint32_t)g + c[2];
    vals[s] = (uint32_t)s;
}

__global__ void k_hist_u32(const uint32_t *keys, uint64_t len, uint32_t *cnt)
{
    uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < len) atomicAdd(&cnt[keys[p]], 1u);
}

int bits_for(uint64_t maxval)
{
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) b++;
    return b;
}

struct Ctx {
    cudaStream_t s;
    DevBuf status;
    ts_status read_status()
    {
        uint32_t st = 0;
        TS_CUDA(cudaMemcpyAsync(&st, status.p, 4, cudaMemcpyDeviceToHost, s));
        TS_CUDA(cudaStreamSynchronize(s));
        if (st & DEV_ERR_INVALID) {
            set_error("invalid database segment (NaN/Inf or t_end <= t_start)");
            return TS_ERR_INVALID_ARG;
        }
        if (st & DEV_ERR_OVERFLOW) {
            set_error("index array longer than 2^32 - 1 entries");
            return TS_ERR_CAPACITY;
        }
        if (st) {
            set_error("index build: device status 0x%x", st);
            return TS_ERR_INTERNAL;
        }
        return TS_OK;
    }
};

// Scan counts into positions and return the total (synchronises; index building is offline).
ts_status counts_to_pos(Ctx &c, const uint32_t *cnt, uint64_t n, DevBuf &pos, uint64_t *total)
{
    TS_CHECK(pos.alloc(sizeof(uint32_t) * (n + 1), c.s));
    TS_CHECK(scan_u32(cnt, pos.as<uint32_t>(), n, c.status.as<uint32_t>(), c.s));
    uint32_t t = 0;
    TS_CUDA(cudaMemcpyAsync(&t, pos.as<uint32_t>() + n, 4, cudaMemcpyDeviceToHost, c.s));
    TS_CHECK(c.read_status());
    *total = t;
    return TS_OK;
}

// One dimension of the spatiotemporal index.
ts_status build_st_dim(Ctx &c, Index *ix, int dim, const double *lo, const double *hi,
                       const uint32_t *bin_of)
{
    const uint64_t n = ix->n;
    const int v = (int)ix->v[dim];
    DevBuf cnt, pos;
    TS_CHECK(cnt.alloc(sizeof(uint32_t) * n, c.s));
    k_part_count<<<nblocks(n), TPB, 0, c.s>>>(lo, hi, n, ix->sub_lo[dim], ix->sub_w[dim], v,
                                              cnt.as<uint32_t>());
    TS_LAUNCHED();
    uint64_t len = 0;
    TS_CHECK(counts_to_pos(c, cnt.as<uint32_t>(), n, pos, &len));
    DevBuf keys;
    TS_CHECK(keys.alloc(sizeof(uint32_t) * len, c.s));
    TS_CHECK(ix->alloc(&ix->st_ids[dim], len));
    k_part_emit<<<nblocks(n), TPB, 0, c.s>>>(lo, hi, n, ix->sub_lo[dim], ix->sub_w[dim], v,
                                             pos.as<uint32_t>(), keys.as<uint32_t>(),
                                             ix->st_ids[dim]);
    TS_LAUNCHED();
    TS_CHECK(radix_sort_u32(keys.as<uint32_t>(), ix->st_ids[dim], len, bits_for((uint64_t)v - 1),
                            c.s));
    uint64_t nbins = (uint64_t)v * ix->m;
    DevBuf h;
    TS_CHECK(h.alloc(sizeof(uint32_t) * nbins, c.s));
    TS_CUDA(cudaMemsetAsync(h.p, 0, sizeof(uint32_t) * nbins, c.s));
    k_st_hist<<<nblocks(len), TPB, 0, c.s>>>(keys.as<uint32_t>(), ix->st_ids[dim], len, bin_of,
                                             ix->m, h.as<uint32_t>());
    TS_LAUNCHED();
    TS_CHECK(ix->alloc(&ix->st_off[dim], nbins + 1));
    TS_CHECK(scan_u32(h.as<uint32_t>(), ix->st_off[dim], nbins, c.status.as<uint32_t>(), c.s));
    TS_CHECK(ix->alloc(&ix->st_rec[dim], len));
    k_gather_rec<<<nblocks(len), TPB, 0, c.s>>>(ix->st_ids[dim], len, ix->rec, ix->st_rec[dim]);
    TS_LAUNCHED();
    ix->st_len[dim] = len;
    return c.read_status();
}

ts_status build_grid(Ctx &c, Index *ix, const double *lo3, const double *hi3)
{
    (void)hi3;
    const uint64_t n = ix->n;
    const int g = (int)ix->g;
    DevBuf keys;
    TS_CHECK(keys.alloc(sizeof(uint32_t) * n, c.s));
    TS_CHECK(ix->alloc(&ix->ga, n));
    k_grid_key<<<nblocks(n), TPB, 0, c.s>>>(lo3, n, ix->g_lo[0], ix->g_lo[1], ix->g_lo[2],
                                            ix->g_w[0], ix->g_w[1], ix->g_w[2], g,
                                            keys.as<uint32_t>(), ix->ga);
    TS_LAUNCHED();
    const uint64_t ncell = (uint64_t)g * g * g;
    TS_CHECK(radix_sort_u32(keys.as<uint32_t>(), ix->ga, n, bits_for(ncell - 1), c.s));
    DevBuf h;
    TS_CHECK(h.alloc(sizeof(uint32_t) * ncell, c.s));
    TS_CUDA(cudaMemsetAsync(h.p, 0, sizeof(uint32_t) * ncell, c.s));
    k_hist_u32<<<nblocks(n), TPB, 0, c.s>>>(keys.as<uint32_t>(), n, h.as<uint32_t>());
    TS_LAUNCHED();
    TS_CHECK(ix->alloc(&ix->g_off, ncell + 1));
    TS_CHECK(scan_u32(h.as<uint32_t>(), ix->g_off, ncell, c.status.as<uint32_t>(), c.s));
    TS_CHECK(ix->alloc(&ix->ga_rec, n));
    k_gather_rec<<<nblocks(n), TPB, 0, c.s>>>(ix->ga, n, ix->rec, ix->ga_rec);
    TS_LAUNCHED();
    // chunk bounding records: the cell sort is stable over the start-time order, so a chunk of
    // a cell spans a short stretch of time and a query's window skips most of a cell's chunks
    const uint64_t nchunks = (n + 63) / 64;
    TS_CHECK(ix->alloc(&ix->gbox, nchunks));
    const unsigned cb = (unsigned)std::min<uint64_t>((nchunks * 32 + TPB - 1) / TPB, 152 * 32);
    k_chunk_box<<<cb, TPB, 0, c.s>>>(ix->ga_rec, n, nchunks, ix->gbox);
    TS_LAUNCHED();
    ix->g_len = n;
    return c.read_status();
}

}  // namespace

void destroy_index(Index *ix)
{
    if (!ix) return;
    cudaDeviceSynchronize();
    for (void *p : ix->allocs) cudaFree(p);
    ix->magic = 0;
    delete ix;
}

// Boundary table lo + j*w (j = 0..v) of a partition, evaluated exactly as part_bound does.
static ts_status upload_bounds(Index *ix, double **dst, double lo, double w, uint32_t v,
                               cudaStream_t s)
{
    std::vector<double> h(v + 1);
    for (uint32_t j = 0; j <= v; j++) h[j] = part_bound(lo, w, (int)j);
    TS_CHECK(ix->alloc(dst, v + 1));
    TS_CUDA(cudaMemcpyAsync(*dst, h.data(), sizeof(double) * (v + 1), cudaMemcpyHostToDevice, s));
    TS_CUDA(cudaStreamSynchronize(s));
    return TS_OK;
}

ts_status build_index(const ts_segments *db, const ts_index_params *p, cudaStream_t s,
                      Index **out)
{
    if (!db || !p || !out) {
        set_error("ts_build_index: NULL argument");
        return TS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (db->n == 0 || db->n > 0x7fffffffull) {
        set_error("ts_build_index: database size %llu outside [1, 2^31 - 1]",
                  (unsigned long long)db->n);
        return TS_ERR_INVALID_ARG;
    }
    if (p->kind < TS_INDEX_BRUTE || p->kind > TS_INDEX_SPATIOTEMPORAL) {
        set_error("ts_build_index: unknown index kind %d", p->kind);
        return TS_ERR_INVALID_ARG;
    }
    if (p->grid_cells > 512) {
        set_error("ts_build_index: grid_cells %u above 512", p->grid_cells);
        return TS_ERR_INVALID_ARG;
    }
    const double *cols[8] = {db->x0, db->y0, db->z0, db->t0, db->x1, db->y1, db->z1, db->t1};
    for (int k = 0; k < 8; k++)
        if (!cols[k]) {
            set_error("ts_build_index: NULL column %d", k);
            return TS_ERR_INVALID_ARG;
        }
    const uint64_t n = db->n;
    Ctx c;
    c.s = s;
    TS_CHECK(c.status.alloc(4, s));
    TS_CUDA(cudaMemsetAsync(c.status.p, 0, 4, s));

    // device copy of the inputs when they live on the host
    DevBuf hostcopy;
    SegIn in;
    if (db->on_host) {
        TS_CHECK(hostcopy.alloc(sizeof(double) * n * 8, s));
        for (int k = 0; k < 8; k++) {
            double *dst = hostcopy.as<double>() + (uint64_t)k * n;
            TS_CUDA(cudaMemcpyAsync(dst, cols[k], sizeof(double) * n, cudaMemcpyHostToDevice, s));
            in.f[k] = dst;
        }
    } else {
        for (int k = 0; k < 8; k++) in.f[k] = cols[k];
    }

    Index *ix = new Index();
    ix->kind = p->kind;
    ix->n = n;
    cudaGetDevice(&ix->device);
    struct Guard {
        Index *&p;
        ~Guard() { if (p) destroy_index(p); }
    } guard{ix};

    // ingest
    DevBuf keys, vals, red;
    TS_CHECK(keys.alloc(sizeof(uint64_t) * n, s));
    TS_CHECK(vals.alloc(sizeof(uint32_t) * n, s));
    TS_CHECK(red.alloc(sizeof(unsigned long long) * R_N, s));
    k_init_red<<<1, 32, 0, s>>>(red.as<unsigned long long>());
    TS_LAUNCHED();
    k_ingest<<<nblocks(n), TPB, 0, s>>>(in, n, keys.as<uint64_t>(), vals.as<uint32_t>(),
                                        red.as<unsigned long long>(), c.status.as<uint32_t>());
    TS_LAUNCHED();
    unsigned long long hred[R_N];
    TS_CUDA(cudaMemcpyAsync(hred, red.p, sizeof(hred), cudaMemcpyDeviceToHost, s));
    TS_CHECK(c.read_status());
    ix->tmin = dkey_inv(hred[R_TMIN]);
    ix->tmax = dkey_inv(hred[R_TMAX]);
    ix->max_dur = dkey_inv(hred[R_DUR]);
    for (int d = 0; d < 3; d++) {
        ix->emin[d] = dkey_inv(hred[R_EMIN + d]);
        ix->emax[d] = dkey_inv(hred[R_EMAX + d]);
        ix->longest[d] = dkey_inv(hred[R_LONG + d]);
    }

    // sort by start time (stable: ties in input order)
    TS_CHECK(radix_sort_u64(keys.as<uint64_t>(), vals.as<uint32_t>(), n, 64, s));
    TS_CHECK(ix->alloc(&ix->seg, n));
    TS_CHECK(ix->alloc(&ix->rec, n));
    TS_CHECK(ix->alloc(&ix->orig, n));
    k_gather<<<nblocks(n), TPB, 0, s>>>(in, n, vals.as<uint32_t>(), ix->seg, ix->rec, ix->orig);
    TS_LAUNCHED();
    keys.release();
    vals.release();

    // temporal bins (all kinds: the schedule of every index starts from the time range)
    {
        uint64_t m = p->t_bins;
        double span = ix->tmax - ix->tmin;
        if (m == 0) {
            double mm = ix->max_dur > 0 ? ceil(4.0 * span / ix->max_dur) : 1.0;
            if (!(mm >= 1.0)) mm = 1.0;
            if (mm > (double)n) mm = (double)n;
            if (mm > 4e6) mm = 4e6;
            m = (uint64_t)mm;
        }
        if (p->kind == TS_INDEX_BRUTE || p->kind == TS_INDEX_SPATIAL) m = 1;
        if (m > 0x3fffffffull) {
            set_error("ts_build_index: t_bins %llu too large", (unsigned long long)m);
            return TS_ERR_INVALID_ARG;
        }
        ix->m = (uint32_t)m;
        ix->b = span / (double)ix->m;
    }
    DevBuf bin_of, end_key;
    TS_CHECK(bin_of.alloc(sizeof(uint32_t) * n, s));
    TS_CHECK(end_key.alloc(sizeof(unsigned long long) * ix->m, s));
    TS_CHECK(ix->alloc(&ix->bin_start, ix->m));
    TS_CHECK(ix->alloc(&ix->bin_end, ix->m));
    TS_CHECK(ix->alloc(&ix->bin_pmax, ix->m));
    TS_CHECK(ix->alloc(&ix->bin_off, (uint64_t)ix->m + 1));
    k_bins_init<<<nblocks(ix->m), TPB, 0, s>>>(ix->m, ix->tmin, ix->b, ix->bin_start,
                                               end_key.as<unsigned long long>());
    TS_LAUNCHED();
    k_bin_of<<<nblocks(n), TPB, 0, s>>>(ix->seg, n, ix->m, ix->tmin, ix->b, bin_of.as<uint32_t>(),
                                        end_key.as<unsigned long long>());
    TS_LAUNCHED();
    k_bin_bounds<<<nblocks(n), TPB, 0, s>>>(bin_of.as<uint32_t>(), n, ix->m, ix->bin_off);
    TS_LAUNCHED();
    k_bin_end_final<<<nblocks(ix->m), TPB, 0, s>>>(end_key.as<unsigned long long>(), ix->m,
                                                   ix->bin_end);
    TS_LAUNCHED();
    k_prefix_max<<<1, 1024, 0, s>>>(ix->bin_end, ix->m, ix->bin_pmax);
    TS_LAUNCHED();

    if (p->kind != TS_INDEX_SPATIAL) {
        // bins ordered by x inside (ranges over the start-time order cover whole bins)
        DevBuf tkeys, tvals;
        TS_CHECK(tkeys.alloc(sizeof(uint64_t) * n, s));
        TS_CHECK(tvals.alloc(sizeof(uint32_t) * n, s));
        k_tx_key<<<nblocks(n), TPB, 0, s>>>(ix->rec, bin_of.as<uint32_t>(), n,
                                            tkeys.as<uint64_t>(), tvals.as<uint32_t>());
        TS_LAUNCHED();
        TS_CHECK(radix_sort_u64(tkeys.as<uint64_t>(), tvals.as<uint32_t>(), n,
                                32 + bits_for((uint64_t)ix->m - 1), s));
        const uint64_t nchunks = (n + 63) / 64;
        TS_CHECK(ix->alloc(&ix->trec, n));
        TS_CHECK(ix->alloc(&ix->tid, n));
        TS_CHECK(ix->alloc(&ix->tbox, nchunks));
        TS_CUDA(cudaMemcpyAsync(ix->tid, tvals.p, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice,
                                s));
        k_gather_rec<<<nblocks(n), TPB, 0, s>>>(ix->tid, n, ix->rec, ix->trec);
        TS_LAUNCHED();
        const unsigned cb = (unsigned)std::min<uint64_t>((nchunks * 32 + TPB - 1) / TPB, 152 * 32);
        k_chunk_box<<<cb, TPB, 0, s>>>(ix->trec, n, nchunks, ix->tbox);
        TS_LAUNCHED();
    }

    if (p->kind == TS_INDEX_SPATIOTEMPORAL || p->kind == TS_INDEX_SPATIAL) {
        DevBuf lo3, hi3;
        TS_CHECK(lo3.alloc(sizeof(double) * n * 3, s));
        TS_CHECK(hi3.alloc(sizeof(double) * n * 3, s));
        for (int d = 0; d < 3; d++) {
            k_mbb<<<nblocks(n), TPB, 0, s>>>(in, ix->orig, n, d, lo3.as<double>() + d * n,
                                             hi3.as<double>() + d * n);
            TS_LAUNCHED();
        }
        if (p->kind == TS_INDEX_SPATIOTEMPORAL) {
            uint32_t v_req = p->sub_bins ? p->sub_bins : 16u;
            for (int d = 0; d < 3; d++) {
                // v lowered so a subbin is at least as wide as the longest entry (Sec. 4.3)
                double ext = ix->emax[d] - ix->emin[d];
                double v = v_req < 1 ? 1.0 : (double)v_req;
                if (ix->longest[d] > 0.0) {
                    double cap = floor(ext / ix->longest[d]);
                    if (cap < 1.0) cap = 1.0;
                    if (v > cap) v = cap;
                }
                if (!(ext > 0.0)) v = 1.0;
                if (v > 4096.0) v = 4096.0;
                ix->v[d] = (uint32_t)v;
                ix->sub_lo[d] = ix->emin[d];
                ix->sub_w[d] = ext / (double)ix->v[d];
                TS_CHECK(upload_bounds(ix, &ix->sub_bound[d], ix->sub_lo[d], ix->sub_w[d],
                                       ix->v[d], s));
                TS_CHECK(build_st_dim(c, ix, d, lo3.as<double>() + d * n, hi3.as<double>() + d * n,
                                      bin_of.as<uint32_t>()));
            }
        } else {
            uint32_t g = p->grid_cells ? p->grid_cells : 50u;
            ix->g = g;
            for (int d = 0; d < 3; d++) {
                ix->g_lo[d] = ix->emin[d];
                ix->g_w[d] = (ix->emax[d] - ix->emin[d]) / (double)g;
                TS_CHECK(upload_bounds(ix, &ix->g_bound[d], ix->g_lo[d], ix->g_w[d], g, s));
            }
            TS_CHECK(build_grid(c, ix, lo3.as<double>(), hi3.as<double>()));
        }
    }
    TS_CHECK(c.read_status());
    *out = ix;
    ix = nullptr;  // disarm the guard
    return TS_OK;
}

}  // namespace ts
