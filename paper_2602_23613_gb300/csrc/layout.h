// Device layouts of the V-cycle: sliced ELL with L lanes per row, and the CTA-chunked layout of
// the Schwarz smoother.  Shared by the kernels and the driver.
#pragma once
#include "common.cuh"

namespace amgh {

constexpr int CTA_THREADS = 256;
constexpr int WARPS_PER_CTA = CTA_THREADS / 32;

// Sliced ELL with L lanes per row.  A slice is 32 lanes = 32/L consecutive rows; entry e of the
// slice's row q lives at slice_ptr[s] + 32 * (e / L) + q * L + e % L.  A warp reading step t of
// its slice touches 32 consecutive values, whatever L is.  Padding: value 0, a valid column.
template <class V>
struct SellL {
    int nrows = 0, nslices = 0, L = 1;
    int64_t stored = 0;
    DevArray<int64_t> slice_ptr;
    DevArray<int32_t> col;
    DevArray<V> val;
};

template <class V>
struct SellLView {
    int nrows, nslices;
    const int64_t* __restrict__ slice_ptr;
    const int32_t* __restrict__ col;
    const V* __restrict__ val;
};

template <class V>
inline SellLView<V> view(const SellL<V>& s) {
    return {s.nrows, s.nslices, s.slice_ptr.p, s.col.p, s.val.p};
}

// words of a grid barrier (count, generation, abort) and the error flag its waits raise
struct GridBarrier {
    unsigned* count;
    unsigned* gen;
    unsigned* abort;
    int* err;
};

// Schwarz smoother of one level.  Stars of one colour are packed, without being split, into
// chunks of SLOTS = 256/L row slots; a chunk is processed by one CTA (L lanes per row slot).  The
// chunk's rows form 8 SELL slices (one per warp); the block inverses are stored per chunk as
// [k][slot] (slot fastest).
template <class V>
struct SmootherL {
    int L = 1, slots = CTA_THREADS, nctas = 0, bmax = 1, ncolours = 0;
    bool fused = false;                       // whole sweep in one single-CTA launch
    int persist = 0;                          // > 0: whole sweep in one cooperative launch of this many CTAs
    bool staged = false;                      // persistent sweep with chunks staged by bulk copies
    bool cluster = false;                     // ... launched as one thread-block cluster
    int cluster2 = 0;                         // > 0: register-prefetching sweep in one cluster of this many CTAs
    int resident = 0;                         // > 0: sweep with x in shared memory, one cluster of this many CTAs
    int resident_g = 1;                       // ... each running this many 256-thread chunk groups
    bool resident_grid = false;               // ... as a cooperative grid of `resident` CTAs, x in global memory
    int n = 0;                                // rows of the level (the resident sweep's copy of x)
    int rs_size = 0, rs_groups = 0;           // shape the resident item lists were built for
    DevArray<int32_t> rs_items;               // per chunk group: (colour step, chunk) pairs in order
    DevArray<int32_t> rs_ptr;                 // chunk group q's items: [rs_ptr[q], rs_ptr[q + 1])
    int stream_grid = 0;                      // > 0: per-colour streaming launches of at most this many CTAs
    bool pdl = false;                         // per-colour launches with programmatic dependent launch
    int stream_bufs = 2;                      // stage buffers per CTA of the streaming launches
    int wmax = 0;                             // longest slice (in 32-wide steps), for the staging buffers
    DevArray<unsigned> bar;                   // count, generation, abort (persistent sweep)
    int* wait_err = nullptr;                  // raised when a barrier wait gives up
    GridBarrier barrier() const { return {bar.p, bar.p + 1, bar.p + 2, wait_err}; }
    std::vector<int32_t> colour_cta_begin;    // host, ncolours + 1
    DevArray<int32_t> colour_cta_begin_d;     // device copy (fused sweep)
    DevArray<int32_t> sweep_d;                // colour sequence 0..C-1, C-2..0 (fused sweep)
    DevArray<int32_t> slot_row;               // nctas * slots, -1 = idle
    DevArray<int16_t> slot_base;              // slot of the star's first row within the chunk
    DevArray<int8_t> slot_bsize;              // rows of the star
    SellL<V> rows;                            // nslices = nctas * 8
    DevArray<V> inv;                          // nctas * bmax * slots
    int64_t stored_rows_nnz = 0;              // algorithmic counts
};

template <class V>
struct SmootherLView {
    int slots, bmax;
    const int32_t* __restrict__ slot_row;
    const int16_t* __restrict__ slot_base;
    const int8_t* __restrict__ slot_bsize;
    SellLView<V> rows;
    const V* __restrict__ inv;
};

template <class V>
inline SmootherLView<V> view(const SmootherL<V>& s) {
    return {s.slots, s.bmax, s.slot_row.p, s.slot_base.p, s.slot_bsize.p, view(s.rows), s.inv.p};
}

// host packing of a level's stars into CTA chunks for a given L
struct StarPacking {
    int L = 1, slots = CTA_THREADS, nctas = 0;
    std::vector<int32_t> colour_cta_begin;
    std::vector<int32_t> slot_row, slot_star;
    std::vector<int16_t> slot_base;
    std::vector<int8_t> slot_bsize;
    std::vector<int32_t> star_cta, star_base;   // per star
};

}  // namespace amgh
