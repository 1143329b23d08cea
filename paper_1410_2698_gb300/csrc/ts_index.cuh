// ts_index.cuh -- the resident index (Sec. 4.1-4.3 re-laid out for HBM).
#pragma once

#include <vector>

#include "ts_internal.cuh"

namespace ts {

constexpr uint32_t MAGIC_INDEX = 0x54534958u;   // "TSIX"
constexpr uint32_t MAGIC_RESULT = 0x54535253u;  // "TSRS"

struct Index {
    uint32_t magic = MAGIC_INDEX;
    int kind = 0;
    uint64_t n = 0;
    int device = 0;

    // entries in start-time order (Sec. 4.2: D sorted by t_start and renumbered)
    SegD *seg = nullptr;     // exact FP64 data
    RecF *rec = nullptr;     // FP32 prefilter records
    uint32_t *orig = nullptr;  // sorted position -> caller's index

    // extents (exact, from the ingest reductions)
    double tmin = 0, tmax = 0, max_dur = 0;
    double emin[3] = {0, 0, 0}, emax[3] = {0, 0, 0}, longest[3] = {0, 0, 0};

    // the entries of every temporal bin once more, ordered by x inside the bin (the bins keep
    // their ranges [B^first, B^last]): records, their start-time positions, and the bounding
    // record of every aligned chunk of 64 (built for every kind whose ranges cover bins)
    RecF *trec = nullptr;
    uint32_t *tid = nullptr;
    RecF *tbox = nullptr;

    // temporal bins (Sec. 4.2)
    uint32_t m = 0;
    double b = 0;
    double *bin_start = nullptr, *bin_end = nullptr, *bin_pmax = nullptr;  // m each
    uint32_t *bin_off = nullptr;  // m + 1

    // spatiotemporal subbins (Sec. 4.3): per dimension an id array in (subbin, bin, time) order,
    // a duplicated prefilter record per id, and offsets off[j*m + i]
    uint32_t v[3] = {0, 0, 0};
    double sub_lo[3] = {0, 0, 0}, sub_w[3] = {0, 0, 0};
    uint32_t *st_ids[3] = {nullptr, nullptr, nullptr};
    RecF *st_rec[3] = {nullptr, nullptr, nullptr};
    uint32_t *st_off[3] = {nullptr, nullptr, nullptr};
    double *sub_bound[3] = {nullptr, nullptr, nullptr};  // lo + j*w for j = 0..v
    uint64_t st_len[3] = {0, 0, 0};

    // flatly structured grid (Sec. 4.1), one cell per entry (the cell of its MBB's minimum
    // corner): dense cell offsets over g^3 cells and the lookup array A with a copy of each
    // entry's prefilter record; inside a cell the entries keep their start-time order, so the
    // bounding records of its chunks are narrow in time
    uint32_t g = 0;
    double g_lo[3] = {0, 0, 0}, g_w[3] = {0, 0, 0};
    uint32_t *ga = nullptr;
    RecF *ga_rec = nullptr;
    RecF *gbox = nullptr;  // bounding record of every aligned chunk of 64 of ga_rec
    uint32_t *g_off = nullptr;  // g^3 + 1
    double *g_bound[3] = {nullptr, nullptr, nullptr};  // lo + j*w for j = 0..g
    uint64_t g_len = 0;

    size_t bytes = 0;
    std::vector<void *> allocs;

    template <class T>
    ts_status alloc(T **p, size_t count)
    {
        size_t nb = sizeof(T) * (count ? count : 1);
        cudaError_t e = cudaMalloc((void **)p, nb);
        if (e != cudaSuccess) {
            *p = nullptr;
            return cuda_status(e, "cudaMalloc(index)");
        }
        allocs.push_back((void *)*p);
        bytes += nb;
        return TS_OK;
    }
};

}  // namespace ts
