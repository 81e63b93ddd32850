// Multiplicative Schwarz on node stars (the OSS-l1 smoother of Section 5): one colour per launch
// over CTA chunks, a whole symmetric sweep of a small level in one single-CTA launch, or a whole
// sweep in one cooperative launch with grid barriers between colours; plus the setup of the chunk
// layout (slot rows, star-block inverses, conditioning estimate).
#include <cuda_bf16.h>

#include <type_traits>

#include "schwarz_chunk.cuh"
#include "star_invert.cuh"
#include "vcycle_kernels.h"

namespace amgh {

namespace {

// Colour step with programmatic dependent launch: the kernel lets its successor launch at once,
// loads everything that does not depend on the previous colour step (slot metadata, the first
// PDL_PREFETCH entries of its row slices, its row of the block inverse), and only then waits for
// the previous kernel's results (griddepcontrol.wait) before gathering x.  The next colour's
// launch and its matrix loads thus overlap this one.  The arithmetic and its order are those of
// schwarz_chunk.  The successor may only launch once every CTA of this grid has started, so the
// head of a chain of such launches always has all its CTAs resident.
constexpr int PDL_PREFETCH = 16;
constexpr int PDL_BMAX = 8;

template <class V, class T, int L>
__global__ void __launch_bounds__(CTA_THREADS) schwarz_pdl_kernel(SmootherLView<V> S, int cta_begin, const T* f,
                                                                  T* x) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    constexpr int SLOTS = CTA_THREADS / L;
    __shared__ T smem_r[CTA_THREADS];
    const int cta = cta_begin + (int)blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, slot = tid / L, sub = tid % L;
    const int64_t gslot = (int64_t)cta * SLOTS + slot;
    const int row = S.slot_row[gslot];
    const int slice = cta * WARPS_PER_CTA + (tid >> 5);
    const int64_t st = S.rows.slice_ptr[slice];
    const int w = (int)((S.rows.slice_ptr[slice + 1] - st) >> 5);
    const int32_t* c = S.rows.col + st + lane;
    const V* v = S.rows.val + st + lane;
    int cc[PDL_PREFETCH];
    V vv[PDL_PREFETCH];
#pragma unroll
    for (int q = 0; q < PDL_PREFETCH; ++q)
        if (q < w) {
            cc[q] = c[32 * q];
            vv[q] = v[32 * q];
        }
    const int base = S.slot_base[gslot], bs = S.slot_bsize[gslot];
    const V* iv = S.inv + (int64_t)cta * S.bmax * SLOTS + slot;
    T ivr[PDL_BMAX];
#pragma unroll
    for (int k = 0; k < PDL_BMAX; ++k) ivr[k] = (sub == 0 && row >= 0 && k < bs) ? widen<T>(iv[(int64_t)k * SLOTS]) : T(0);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    T s = T(0);
#pragma unroll
    for (int q = 0; q < PDL_PREFETCH; ++q)
        if (q < w) s = fma(widen<T>(vv[q]), x[cc[q]], s);
#pragma unroll 8
    for (int t = PDL_PREFETCH; t < w; ++t) s = fma(widen<T>(v[32 * t]), x[c[32 * t]], s);
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (sub == 0) smem_r[slot] = row >= 0 ? f[row] - s : T(0);
    __syncthreads();
    if (sub == 0 && row >= 0) {
        T d = T(0);
#pragma unroll
        for (int k = 0; k < PDL_BMAX; ++k)
            if (k < bs) d = fma(ivr[k], smem_r[base + k], d);
        for (int k = PDL_BMAX; k < bs; ++k) d = fma(widen<T>(iv[(int64_t)k * SLOTS]), smem_r[base + k], d);
        x[row] += d;
    }
}

// Whole sweep in one thread-block cluster of 512-thread CTAs, each running two chunk groups of
// 256 threads (CTA r, group g owns chunk cbeg[c] + 2 r + g of colour c, so the cluster covers
// colours of up to 2 x cluster-size chunks).  Before each hardware cluster barrier every thread
// loads, for its chunk of the next colour step, its slot metadata, the first CL_PREFETCH entries
// of its row slice and its row of the block inverse, into registers; after the barrier only the
// x gathers, the lane reduction and the block solve remain.  The groups synchronise with named
// barriers.  No thread waits on anything but the cluster barrier, which every thread reaches the
// same number of times.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

constexpr int CL_PREFETCH = 16;
constexpr int CL_BMAX = 16;

template <class V, class T, int L>
struct ClusterStep {
    int row = -1, base = 0, bs = 0, w = 0;
    const int32_t* c = nullptr;
    const V* v = nullptr;
    int cc[CL_PREFETCH];
    V vv[CL_PREFETCH];
    T ivr[CL_BMAX];
};

template <class V, class T, int L>
__device__ __forceinline__ void cluster_prefetch(const SmootherLView<V>& S, int cta, bool have, int gtid,
                                                 ClusterStep<V, T, L>& P) {
    constexpr int SLOTS = CTA_THREADS / L;
    const int lane = gtid & 31, slot = gtid / L, sub = gtid % L;
    P.row = -1;
    P.w = 0;
    P.bs = 0;
    if (!have) return;
    const int64_t gslot = (int64_t)cta * SLOTS + slot;
    P.row = S.slot_row[gslot];
    P.base = S.slot_base[gslot];
    P.bs = S.slot_bsize[gslot];
    const int slice = cta * WARPS_PER_CTA + (gtid >> 5);
    const int64_t st = S.rows.slice_ptr[slice];
    P.w = (int)((S.rows.slice_ptr[slice + 1] - st) >> 5);
    P.c = S.rows.col + st + lane;
    P.v = S.rows.val + st + lane;
#pragma unroll
    for (int q = 0; q < CL_PREFETCH; ++q)
        if (q < P.w) {
            P.cc[q] = P.c[32 * q];
            P.vv[q] = P.v[32 * q];
        }
    const V* iv = S.inv + (int64_t)cta * S.bmax * SLOTS + slot;
#pragma unroll
    for (int k = 0; k < CL_BMAX; ++k)
        P.ivr[k] = (sub == 0 && P.row >= 0 && k < P.bs) ? widen<T>(iv[(int64_t)k * SLOTS]) : T(0);
}

__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(CTA_THREADS) : "memory");
}

template <class V, class T, int L>
__global__ void __launch_bounds__(2 * CTA_THREADS, 1) schwarz_cluster2_kernel(SmootherLView<V> S,
                                                                             const int32_t* __restrict__ sweep,
                                                                             int nsteps,
                                                                             const int32_t* __restrict__ cbeg,
                                                                             const T* f, T* x) {
    constexpr int SLOTS = CTA_THREADS / L;
    __shared__ T smem_r[2][CTA_THREADS];
    const int g = threadIdx.x / CTA_THREADS, gtid = threadIdx.x % CTA_THREADS;
    const int lane = gtid & 31, slot = gtid / L, sub = gtid % L;
    const int q = 2 * (int)blockIdx.x + g;
    ClusterStep<V, T, L> P;
    {
        const int c0 = sweep[0], cta0 = cbeg[c0] + q;
        cluster_prefetch<V, T, L>(S, cta0, cta0 < cbeg[c0 + 1], gtid, P);
    }
    for (int st = 0; st < nsteps; ++st) {
        const int c = sweep[st], cta = cbeg[c] + q;
        if (cta < cbeg[c + 1]) {
            T s = T(0);
#pragma unroll
            for (int t = 0; t < CL_PREFETCH; ++t)
                if (t < P.w) s = fma(widen<T>(P.vv[t]), x[P.cc[t]], s);
#pragma unroll 8
            for (int t = CL_PREFETCH; t < P.w; ++t) s = fma(widen<T>(P.v[32 * t]), x[P.c[32 * t]], s);
#pragma unroll
            for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (sub == 0) smem_r[g][slot] = P.row >= 0 ? f[P.row] - s : T(0);
            group_sync(g);
            if (sub == 0 && P.row >= 0) {
                T d = T(0);
#pragma unroll
                for (int k = 0; k < CL_BMAX; ++k)
                    if (k < P.bs) d = fma(P.ivr[k], smem_r[g][P.base + k], d);
                x[P.row] += d;
            }
            group_sync(g);
        }
        if (st + 1 < nsteps) {
            const int cn = sweep[st + 1], ctan = cbeg[cn] + q;
            cluster_prefetch<V, T, L>(S, ctan, ctan < cbeg[cn + 1], gtid, P);
            __syncthreads();
            cluster_sync_all();
        }
    }
}

// Whole symmetric sweep of a small level: colours in sweep order, chunks of a colour in turn, one
// CTA; the barriers inside schwarz_chunk order every colour after the previous one (x is read
// with ordinary coherent loads).
template <class V, class T, int L>
__global__ void __launch_bounds__(CTA_THREADS) schwarz_fused_kernel(SmootherLView<V> S, const int32_t* __restrict__ sweep,
                                                                    int nsteps, const int32_t* __restrict__ cbeg,
                                                                    const T* f, T* x) {
    __shared__ T smem_r[CTA_THREADS];
    for (int st = 0; st < nsteps; ++st) {
        const int c = sweep[st];
        for (int cta = cbeg[c]; cta < cbeg[c + 1]; ++cta) schwarz_chunk<V, T, L>(S, cta, f, x, smem_r);
    }
}

// Grid-wide barrier of a cooperative launch.  A CTA arrives with one atomic after a fence over
// its writes; the last of the grid's arrivals resets the count and advances the generation word.
// Waits are bounded: a CTA that polls SPIN_LIMIT times raises the abort word and the error flag
// and gives up, and every waiting CTA that sees the abort word gives up at once, so a grid whose
// CTAs were not all resident ends with an error instead of hanging.
constexpr long long SPIN_LIMIT = 1ll << 20;   // about a second of polling

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_sync(const GridBarrier& b, unsigned& gen, unsigned arrivals) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        __threadfence();
        if (atomicAdd(b.count, 1u) == arrivals - 1) {
            atomicExch(b.count, 0u);
            __threadfence();
            atomicExch(b.gen, gen + 1);
        } else {
            long long it = 0;
            while (ld_acquire_gpu(b.gen) == gen) {
                if (ld_acquire_gpu(b.abort) != 0u) { good = 0; break; }
                if (++it > SPIN_LIMIT) {
                    atomicExch(b.abort, 1u);
                    atomicExch(b.err, 1);
                    good = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        gen += 1;
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Whole symmetric sweep of a level in one cooperative launch: the chunks of a colour are spread
// over the grid, and a grid barrier orders each colour after the previous one.
template <class V, class T, int L>
__global__ void __launch_bounds__(CTA_THREADS) schwarz_persistent_kernel(SmootherLView<V> S,
                                                                         const int32_t* __restrict__ sweep, int nsteps,
                                                                         const int32_t* __restrict__ cbeg, const T* f,
                                                                         T* x, GridBarrier bar) {
    __shared__ T smem_r[CTA_THREADS];
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = ld_acquire_gpu(bar.gen);   // cannot advance before this CTA arrives
    for (int st = 0; st < nsteps; ++st) {
        const int c = sweep[st];
        for (int cta = cbeg[c] + (int)blockIdx.x; cta < cbeg[c + 1]; cta += (int)gridDim.x)
            schwarz_chunk<V, T, L>(S, cta, f, x, smem_r);
        if (st + 1 < nsteps && !grid_sync(bar, gen, gridDim.x)) return;
    }
}

// Self-test of the bounded waits: a grid barrier that expects one arrival more than the grid
// has can never complete, so every CTA's wait must give up, raise *b.err and return.
__global__ void wait_timeout_probe_kernel(GridBarrier b) {
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = ld_acquire_gpu(b.gen);
    grid_sync(b, gen, gridDim.x + 1);
}

// ---------------------------------------------------------------------------------------------
// Staged persistent sweep: a CTA owns at most one chunk per colour step (grid >= the largest
// colour's chunk count).  The chunk's SELL slices (columns, values) and block inverses are one
// contiguous range each, so one thread copies them into shared memory with three bulk async
// copies that complete on an mbarrier.  The copies for step s+1 are issued at the start of step
// s (double buffer), so after a grid barrier only the x gathers, the residual reduction and the
// block solve remain on the critical path.  mbarrier waits are bounded like the grid barrier.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bytes must be a multiple of 16 and both addresses 16-byte aligned (checked by the host layout)
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// shared-memory layout of one stage buffer of a chunk
template <class V>
struct StageLayout {
    int64_t elems;      // 8 slices x 32 lanes x wmax
    int64_t inv_elems;  // bmax x slots
    __host__ __device__ int64_t col_bytes() const { return elems * 4; }
    __host__ __device__ int64_t val_bytes() const { return elems * (int64_t)sizeof(V); }
    __host__ __device__ int64_t inv_bytes() const { return inv_elems * (int64_t)sizeof(V); }
    __host__ __device__ int64_t stage_bytes() const {
        return (col_bytes() + val_bytes() + inv_bytes() + 15) / 16 * 16;
    }
};

template <class V>
__device__ __forceinline__ void stage_issue(const SmootherLView<V>& S, const StageLayout<V>& lay, int cta,
                                            unsigned char* buf, uint64_t* bar) {
    const int64_t s0 = S.rows.slice_ptr[(int64_t)cta * WARPS_PER_CTA];
    const int64_t s1 = S.rows.slice_ptr[(int64_t)cta * WARPS_PER_CTA + WARPS_PER_CTA];
    const uint32_t n = (uint32_t)(s1 - s0);
    const uint32_t cb = n * 4u, vb = n * (uint32_t)sizeof(V), ib = (uint32_t)lay.inv_bytes();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, cb + vb + ib);
    bulk_copy_g2s(buf, S.rows.col + s0, cb, bar);
    bulk_copy_g2s(buf + lay.col_bytes(), S.rows.val + s0, vb, bar);
    bulk_copy_g2s(buf + lay.col_bytes() + lay.val_bytes(), S.inv + (int64_t)cta * lay.inv_elems, ib, bar);
}

// bounded wait on a stage buffer; false (after raising the abort word and the error flag) when
// the wait gives up
__device__ __forceinline__ bool stage_wait(uint64_t* bar, uint32_t parity, const GridBarrier& gb) {
    long long it = 0;
    while (!mbar_test_wait(bar, parity)) {
        if (++it > SPIN_LIMIT) {
            atomicExch(gb.abort, 1u);
            atomicExch(gb.err, 1);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}


// CLUSTER: the grid is one thread-block cluster and the colour steps are ordered by the hardware
// cluster barrier instead of the bounded grid barrier.  A CTA whose bounded copy wait gives up
// stops computing and copying but keeps arriving at every cluster barrier, so the others finish.
template <class V, class T, int L, bool CLUSTER>
__global__ void __launch_bounds__(CTA_THREADS) schwarz_staged_kernel(SmootherLView<V> S, StageLayout<V> lay,
                                                                     const int32_t* __restrict__ sweep, int nsteps,
                                                                     const int32_t* __restrict__ cbeg, const T* f,
                                                                     T* x, GridBarrier bar) {
    constexpr int SLOTS = CTA_THREADS / L;
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ T smem_r[CTA_THREADS];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ int stop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, slot = tid / L, sub = tid % L;
    const int64_t sbytes = lay.stage_bytes();
    if (tid == 0) {
        mbar_init(&mbar[0]);
        mbar_init(&mbar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stop = 0;
    }
    __syncthreads();
    uint32_t parity = 0u, pending = 0u;   // bit b: phase parity / copy in flight of stage buffer b
    unsigned gen = 0;
    if (tid == 0) gen = ld_acquire_gpu(bar.gen);
    {
        const int c0 = sweep[0], cta0 = cbeg[c0] + (int)blockIdx.x;
        if (cta0 < cbeg[c0 + 1]) {
            if (tid == 0) stage_issue<V>(S, lay, cta0, dyn, &mbar[0]);
            pending |= 1u;
        }
    }
    for (int st = 0; st < nsteps; ++st) {
        const int b = st & 1;
        unsigned char* sb = dyn + b * sbytes;
        const int c = sweep[st], cta = cbeg[c] + (int)blockIdx.x;
        if (st + 1 < nsteps && !(CLUSTER && stop)) {
            const int cn = sweep[st + 1], ctan = cbeg[cn] + (int)blockIdx.x;
            if (ctan < cbeg[cn + 1]) {
                if (tid == 0) stage_issue<V>(S, lay, ctan, dyn + (b ^ 1) * sbytes, &mbar[b ^ 1]);
                pending |= 2u >> b;
            }
        }
        if (cta < cbeg[c + 1] && !(CLUSTER && stop)) {
            // per-slot metadata and slice offsets do not depend on x
            const int64_t gslot = (int64_t)cta * SLOTS + slot;
            const int row = S.slot_row[gslot];
            const int base = S.slot_base[gslot], bs = S.slot_bsize[gslot];
            const int64_t s0 = S.rows.slice_ptr[(int64_t)cta * WARPS_PER_CTA];
            const int64_t st0 = S.rows.slice_ptr[(int64_t)cta * WARPS_PER_CTA + warp];
            const int w = (int)((S.rows.slice_ptr[(int64_t)cta * WARPS_PER_CTA + warp + 1] - st0) >> 5);
            const bool ok = stage_wait(&mbar[b], (parity >> b) & 1u, bar);
            if (!ok) {
                stop = 1;   // the copy stays pending: drained (bounded) below
            } else {
                parity ^= 1u << b;
                pending &= ~(1u << b);
            }
            __syncthreads();
            if (stop) {
                if (!CLUSTER) break;
            } else {
            const int32_t* scol = reinterpret_cast<const int32_t*>(sb) + (st0 - s0) + lane;
            const V* sval = reinterpret_cast<const V*>(sb + lay.col_bytes()) + (st0 - s0) + lane;
            const V* sinv = reinterpret_cast<const V*>(sb + lay.col_bytes() + lay.val_bytes());
            T s = T(0);
#pragma unroll 8
            for (int t = 0; t < w; ++t) s = fma(widen<T>(sval[32 * t]), x[scol[32 * t]], s);
#pragma unroll
            for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (sub == 0) smem_r[slot] = row >= 0 ? f[row] - s : T(0);
            __syncthreads();
            if (sub == 0 && row >= 0) {
                T d = T(0);
                for (int k = 0; k < bs; ++k) d = fma(widen<T>(sinv[k * SLOTS + slot]), smem_r[base + k], d);
                x[row] += d;
            }
            }
        }
        if (st + 1 < nsteps) {
            if (CLUSTER) {
                __syncthreads();
                cluster_sync_all();
            } else if (!grid_sync(bar, gen, gridDim.x)) {
                break;
            }
        }
    }
    // leave no bulk copy in flight into this CTA's shared memory
    for (int q = 0; q < 2; ++q)
        if ((pending >> q) & 1u) stage_wait(&mbar[q], (parity >> q) & 1u, bar);
}

// ---------------------------------------------------------------------------------------------
// Streaming colour step: one launch per colour; each CTA walks the colour's chunks
// (blockIdx.x, + gridDim.x, ...) with the chunk's SELL columns and values double-buffered in
// shared memory by bulk async copies, so the matrix stream runs at copy speed while the previous
// chunk computes.  No CTA waits on another; the mbarrier waits are bounded and raise *err.
// ---------------------------------------------------------------------------------------------
template <class V>
__device__ __forceinline__ void stream_issue(const SmootherLView<V>& S, int64_t col_bytes_cap, int cta,
                                             unsigned char* buf, uint64_t* bar) {
    const int64_t s0 = S.rows.slice_ptr[(int64_t)cta * WARPS_PER_CTA];
    const int64_t s1 = S.rows.slice_ptr[(int64_t)cta * WARPS_PER_CTA + WARPS_PER_CTA];
    const uint32_t n = (uint32_t)(s1 - s0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, n * (4u + (uint32_t)sizeof(V)));
    bulk_copy_g2s(buf, S.rows.col + s0, n * 4u, bar);
    bulk_copy_g2s(buf + col_bytes_cap, S.rows.val + s0, n * (uint32_t)sizeof(V), bar);
}

__device__ __forceinline__ bool stream_wait(uint64_t* bar, uint32_t parity, int* err) {
    long long it = 0;
    while (!mbar_test_wait(bar, parity)) {
        if (++it > SPIN_LIMIT) {
            atomicExch(err, 1);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

constexpr int STREAM_BMAX = 8;   // block rows held in registers by the streaming kernel

template <class V, class T, int L, int NBUF>
__global__ void __launch_bounds__(CTA_THREADS) schwarz_stream_kernel(SmootherLView<V> S, int64_t elems, int cbeg,
                                                                     int cend, const T* f, T* x, int* err) {
    constexpr int SLOTS = CTA_THREADS / L;
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ T smem_r[CTA_THREADS];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ int stop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, slot = tid / L, sub = tid % L;
    const int64_t col_bytes = elems * 4, sbytes = (elems * (4 + (int64_t)sizeof(V)) + 15) / 16 * 16;
    if (tid == 0) {
        mbar_init(&mbar[0]);
        mbar_init(&mbar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stop = 0;
    }
    __syncthreads();
    uint32_t parity = 0u, pending = 0u;
    int cta = cbeg + (int)blockIdx.x;
    if (NBUF == 2 && cta < cend) {
        if (tid == 0) stream_issue<V>(S, col_bytes, cta, dyn, &mbar[0]);
        pending = 1u;
    }
    for (int k = 0; cta < cend; ++k, cta += (int)gridDim.x) {
        const int b = NBUF == 2 ? (k & 1) : 0;
        unsigned char* sb = dyn + b * sbytes;
        if (NBUF == 2) {
            // the next chunk's copy overlaps this chunk's compute
            const int nxt = cta + (int)gridDim.x;
            if (nxt < cend) {
                if (tid == 0) stream_issue<V>(S, col_bytes, nxt, dyn + (b ^ 1) * sbytes, &mbar[b ^ 1]);
                pending |= 2u >> b;
            }
        } else {
            // one buffer: the copy overlaps the other CTAs on the SM
            if (tid == 0) stream_issue<V>(S, col_bytes, cta, dyn, &mbar[0]);
            pending = 1u;
        }
        // everything that does not depend on the staged data or on x, ahead of the wait
        const int64_t gslot = (int64_t)cta * SLOTS + slot;
        const int row = S.slot_row[gslot];
        const int base = S.slot_base[gslot], bs = S.slot_bsize[gslot];
        const int64_t s0 = S.rows.slice_ptr[(int64_t)cta * WARPS_PER_CTA];
        const int64_t st0 = S.rows.slice_ptr[(int64_t)cta * WARPS_PER_CTA + warp];
        const int w = (int)((S.rows.slice_ptr[(int64_t)cta * WARPS_PER_CTA + warp + 1] - st0) >> 5);
        const T fr = (sub == 0 && row >= 0) ? f[row] : T(0);
        T ivr[STREAM_BMAX];
        const V* iv = S.inv + (int64_t)cta * S.bmax * SLOTS + slot;
#pragma unroll
        for (int q = 0; q < STREAM_BMAX; ++q) ivr[q] = (sub == 0 && q < bs) ? widen<T>(iv[(int64_t)q * SLOTS]) : T(0);
        if (!stream_wait(&mbar[b], (parity >> b) & 1u, err)) stop = 1;
        else {
            parity ^= 1u << b;
            pending &= ~(1u << b);
        }
        __syncthreads();
        if (stop) break;
        const int32_t* scol = reinterpret_cast<const int32_t*>(sb) + (st0 - s0) + lane;
        const V* sval = reinterpret_cast<const V*>(sb + col_bytes) + (st0 - s0) + lane;
        T s = T(0);
#pragma unroll 8
        for (int t = 0; t < w; ++t) s = fma(widen<T>(sval[32 * t]), x[scol[32 * t]], s);
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (sub == 0) smem_r[slot] = row >= 0 ? fr - s : T(0);
        __syncthreads();
        if (sub == 0 && row >= 0) {
            T d = T(0);
#pragma unroll
            for (int q = 0; q < STREAM_BMAX; ++q)
                if (q < bs) d = fma(ivr[q], smem_r[base + q], d);
            x[row] += d;
        }
        __syncthreads();   // the buffer of this chunk is refilled two chunks later
    }
    for (int q = 0; q < 2; ++q)
        if ((pending >> q) & 1u) stream_wait(&mbar[q], (parity >> q) & 1u, err);
}

// ---------------------------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------------------------
template <class V>
__global__ void slotL_fill_kernel(int nctas, int L, const int32_t* __restrict__ slot_row, const int32_t* __restrict__ ptr,
                                  const int32_t* __restrict__ idx, const double* __restrict__ val,
                                  const int64_t* __restrict__ sptr, int32_t* __restrict__ scol, V* __restrict__ sval) {
    const int cta = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    if (cta >= nctas) return;
    const int slots = CTA_THREADS / L;
    const int row = slot_row[(int64_t)cta * slots + tid / L], sub = tid % L;
    const int slice = cta * WARPS_PER_CTA + (tid >> 5);
    const int64_t st = sptr[slice];
    const int w = (int)((sptr[slice + 1] - st) >> 5);
    int b = 0, len = 0;
    if (row >= 0) { b = ptr[row]; len = ptr[row + 1] - b; }
    for (int t = 0; t < w; ++t) {
        const int e = t * L + sub;
        const int64_t o = st + 32 * (int64_t)t + lane;
        if (e < len) { scol[o] = idx[b + e]; sval[o] = narrow<V>(val[b + e]); }
        else { scol[o] = row >= 0 ? row : 0; sval[o] = narrow<V>(0.0); }
    }
}

template <class V>
__global__ void star_inverseL_kernel(const int32_t* __restrict__ Aptr, const int32_t* __restrict__ Aidx,
                                     const double* __restrict__ Aval, int nstars, const int32_t* __restrict__ star_ptr,
                                     const int32_t* __restrict__ star_idx, const int32_t* __restrict__ star_cta,
                                     const int32_t* __restrict__ star_base, int slots, int bmax, V* __restrict__ inv,
                                     int* err_flag) {
    __shared__ double sm[2][2][32 * 33];
    __shared__ double fac[2][32];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * 2 + wl;
    if (j >= nstars) return;
    const int b0 = star_ptr[j], b = star_ptr[j + 1] - b0;
    if (b == 0) return;
    const bool ok = star_invert(Aptr, Aidx, Aval, star_idx, b0, b, sm[wl][0], sm[wl][1], fac[wl]);
    if (!ok && lane == 0) atomicExch(err_flag, 1);
    const int cta = star_cta[j], base = star_base[j];
    if (lane < b)
        for (int k = 0; k < b; ++k)
            inv[((int64_t)cta * bmax + k) * slots + base + lane] = narrow<V>(sm[wl][1][lane * 33 + k]);
}

// small stars (at most 8 rows, e.g. the finest level's node stars): eight warps per CTA with
// 8 x 9 blocks, the same Gauss-Jordan as above
template <class V>
__global__ void __launch_bounds__(256) star_inverse_small_kernel(
    const int32_t* __restrict__ Aptr, const int32_t* __restrict__ Aidx, const double* __restrict__ Aval, int nstars,
    const int32_t* __restrict__ star_ptr, const int32_t* __restrict__ star_idx, const int32_t* __restrict__ star_cta,
    const int32_t* __restrict__ star_base, int slots, int bmax, V* __restrict__ inv, int* err_flag) {
    __shared__ double sm[8][2][8 * 9];
    __shared__ double fac[8][8];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * 8 + wl;
    if (j >= nstars) return;
    const int b0 = star_ptr[j], b = star_ptr[j + 1] - b0;
    if (b == 0) return;
    const bool ok = star_invert_s<9>(Aptr, Aidx, Aval, star_idx, b0, b, sm[wl][0], sm[wl][1], fac[wl]);
    if (!ok && lane == 0) atomicExch(err_flag, 1);
    const int cta = star_cta[j], base = star_base[j];
    if (lane < b)
        for (int k = 0; k < b; ++k)
            inv[((int64_t)cta * bmax + k) * slots + base + lane] = narrow<V>(sm[wl][1][lane * 9 + k]);
}

__global__ void star_kappa_kernel(const int32_t* __restrict__ Aptr, const int32_t* __restrict__ Aidx,
                                  const double* __restrict__ Aval, int nstars, const int32_t* __restrict__ star_ptr,
                                  const int32_t* __restrict__ star_idx, unsigned long long* kappa_bits, int* err_flag) {
    __shared__ double sm[2][2][32 * 33];
    __shared__ double fac[2][32];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * 2 + wl;
    if (j >= nstars) return;
    const int b0 = star_ptr[j], b = star_ptr[j + 1] - b0;
    if (b == 0) return;
    double* M = sm[wl][0];
    double* I = sm[wl][1];
    const bool ok = star_invert(Aptr, Aidx, Aval, star_idx, b0, b, M, I, fac[wl]);
    if (!ok && lane == 0) atomicExch(err_flag, 1);
    // 1-norms: lane c sums column c of the inverse, and of A_BB re-read from A (M now holds I)
    double acol = 0.0, icol = 0.0;
    if (lane < b) {
        for (int r = 0; r < b; ++r) icol += fabs(I[r * 33 + lane]);
        const int g = star_idx[b0 + lane];   // column lane of A_BB = row lane (symmetric)
        for (int q = Aptr[g]; q < Aptr[g + 1]; ++q)
            if (bsearch_i32(star_idx, b0, b0 + b, Aidx[q]) >= 0) acol += fabs(Aval[q]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        acol = fmax(acol, __shfl_xor_sync(0xffffffffu, acol, o));
        icol = fmax(icol, __shfl_xor_sync(0xffffffffu, icol, o));
    }
    if (lane == 0) {
        const double kap = acol * icol;
        atomicMax(kappa_bits, (unsigned long long)__double_as_longlong(kap));   // positive doubles order as integers
    }
}

template <class V, class T, int L>
void launch_colour_impl(const SmootherL<V>& S, int cb, int ce, const T* f, T* x, cudaStream_t s) {
    if (S.pdl) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(ce - cb));
        cfg.blockDim = dim3(CTA_THREADS);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        AMGH_CUDA(cudaLaunchKernelEx(&cfg, schwarz_pdl_kernel<V, T, L>, view(S), cb, f, x));
        return;
    }
    schwarz_cta_kernel<V, T, L><<<ce - cb, CTA_THREADS, 0, s>>>(view(S), cb, f, x);
}

template <class V, class T, int L>
void launch_fused_impl(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s) {
    schwarz_fused_kernel<V, T, L><<<1, CTA_THREADS, 0, s>>>(view(S), S.sweep_d.p, (int)S.sweep_d.n,
                                                             S.colour_cta_begin_d.p, f, x);
}

template <class V, class T, int L>
void launch_persistent_impl(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)S.persist);
    cfg.blockDim = dim3(CTA_THREADS);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    AMGH_CUDA(cudaLaunchKernelEx(&cfg, schwarz_persistent_kernel<V, T, L>, view(S), (const int32_t*)S.sweep_d.p,
                                 (int)S.sweep_d.n, (const int32_t*)S.colour_cta_begin_d.p, f, x, S.barrier()));
}

__global__ void coop_probe_kernel(int* out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *out = 1;
}

template <class V>
StageLayout<V> stage_layout(const SmootherL<V>& S) {
    StageLayout<V> lay;
    lay.elems = (int64_t)WARPS_PER_CTA * 32 * S.wmax;
    lay.inv_elems = (int64_t)S.bmax * S.slots;
    return lay;
}

template <class V, class T, int L>
void launch_staged_impl(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s) {
    // one chunk per CTA and colour step: refuse a grid smaller than a colour
    for (int c = 0; c < S.ncolours; ++c)
        if (S.colour_cta_begin[c + 1] - S.colour_cta_begin[c] > S.persist)
            throw CudaError{cudaErrorInvalidConfiguration, "staged sweep grid smaller than a colour"};
    const StageLayout<V> lay = stage_layout(S);
    const size_t smem = 2 * (size_t)lay.stage_bytes();   // opt-in limit set by schwarz_staged_cap
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)S.persist);
    cfg.blockDim = dim3(CTA_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (S.cluster) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)S.persist;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
    } else {
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (S.cluster)
        AMGH_CUDA(cudaLaunchKernelEx(&cfg, schwarz_staged_kernel<V, T, L, true>, view(S), lay,
                                     (const int32_t*)S.sweep_d.p, (int)S.sweep_d.n,
                                     (const int32_t*)S.colour_cta_begin_d.p, f, x, S.barrier()));
    else
        AMGH_CUDA(cudaLaunchKernelEx(&cfg, schwarz_staged_kernel<V, T, L, false>, view(S), lay,
                                     (const int32_t*)S.sweep_d.p, (int)S.sweep_d.n,
                                     (const int32_t*)S.colour_cta_begin_d.p, f, x, S.barrier()));
}

// whether one cluster of `size` CTAs of the staged kernel can be resident with this shared memory
template <class V, class T, int L>
bool staged_cluster_ok_impl(int size, size_t smem) {
    int dev = 0, maxsm = 0;
    AMGH_CUDA(cudaGetDevice(&dev));
    AMGH_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (size < 1 || size > 16 || smem + 4096 > (size_t)maxsm) return false;
    auto kern = schwarz_staged_kernel<V, T, L, true>;
    AMGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm - 4096));
    if (size > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)size);
    cfg.blockDim = dim3(CTA_THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters >= 1;
}

template <class V, class T, int L>
int staged_cap_impl(size_t smem) {
    auto kern = schwarz_staged_kernel<V, T, L, false>;
    int dev = 0, nsm = 0, per_sm = 0, maxsm = 0;
    AMGH_CUDA(cudaGetDevice(&dev));
    AMGH_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    AMGH_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (smem + 4096 > (size_t)maxsm) return 0;   // static shared memory needs the rest
    // the opt-in limit is per kernel: raise it to the device's maximum once, so that levels of
    // different staging sizes can share one instantiation
    AMGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm - 4096));
    AMGH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CTA_THREADS, smem));
    return nsm * per_sm;
}

template <class V>
int64_t stream_elems(const SmootherL<V>& S) { return (int64_t)WARPS_PER_CTA * 32 * S.wmax; }
template <class V>
size_t stream_smem(const SmootherL<V>& S, int nbuf) {
    return (size_t)nbuf * (size_t)((stream_elems(S) * (4 + (int64_t)sizeof(V)) + 15) / 16 * 16);
}

template <class V, class T, int L>
void launch_stream_impl(const SmootherL<V>& S, int cb, int ce, const T* f, T* x, cudaStream_t s) {
    const int grid = std::min(ce - cb, S.stream_grid);
    if (S.stream_bufs == 1)
        schwarz_stream_kernel<V, T, L, 1><<<grid, CTA_THREADS, stream_smem(S, 1), s>>>(view(S), stream_elems(S), cb,
                                                                                      ce, f, x, S.wait_err);
    else
        schwarz_stream_kernel<V, T, L, 2><<<grid, CTA_THREADS, stream_smem(S, 2), s>>>(view(S), stream_elems(S), cb,
                                                                                      ce, f, x, S.wait_err);
}

template <class V, class T, int L, int NBUF>
int stream_cap_impl(size_t smem) {
    int dev = 0, nsm = 0, per_sm = 0, maxsm = 0;
    AMGH_CUDA(cudaGetDevice(&dev));
    AMGH_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    AMGH_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (smem + 4096 > (size_t)maxsm) return 0;
    AMGH_CUDA(cudaFuncSetAttribute(schwarz_stream_kernel<V, T, L, NBUF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   maxsm - 4096));
    AMGH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, schwarz_stream_kernel<V, T, L, NBUF>,
                                                            CTA_THREADS, smem));
    return nsm * per_sm;
}

template <class V, class T, int L>
void launch_cluster2_impl(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s) {
    // each of the cluster's 2 x size chunk groups owns one chunk per colour step: refuse a cluster
    // that would leave chunks of some colour unprocessed
    for (int c = 0; c < S.ncolours; ++c)
        if (S.colour_cta_begin[c + 1] - S.colour_cta_begin[c] > 2 * S.cluster2)
            throw CudaError{cudaErrorInvalidConfiguration, "cluster sweep smaller than a colour"};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)S.cluster2);
    cfg.blockDim = dim3(2 * CTA_THREADS);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)S.cluster2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    AMGH_CUDA(cudaLaunchKernelEx(&cfg, schwarz_cluster2_kernel<V, T, L>, view(S), (const int32_t*)S.sweep_d.p,
                                 (int)S.sweep_d.n, (const int32_t*)S.colour_cta_begin_d.p, f, x));
}

template <class V, class T, int L>
bool cluster2_ok_impl(int size) {
    if (size < 1 || size > 8) return false;
    auto kern = schwarz_cluster2_kernel<V, T, L>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)size);
    cfg.blockDim = dim3(2 * CTA_THREADS);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters >= 1;
}

template <class V, class T, int L>
int persistent_cap_impl() {
    int dev = 0, nsm = 0, per_sm = 0;
    AMGH_CUDA(cudaGetDevice(&dev));
    AMGH_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    AMGH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, schwarz_persistent_kernel<V, T, L>,
                                                            CTA_THREADS, 0));
    return nsm * per_sm;
}

}  // namespace

template <class V, class T>
void launch_schwarz_persistent(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s) {
    if (S.resident > 0) {
        launch_schwarz_resident<V, T>(S, f, x, s);
        return;
    }
    if (S.cluster2 > 0) {
        switch (S.L) {
            case 1: launch_cluster2_impl<V, T, 1>(S, f, x, s); break;
            case 2: launch_cluster2_impl<V, T, 2>(S, f, x, s); break;
            case 4: launch_cluster2_impl<V, T, 4>(S, f, x, s); break;
            case 8: launch_cluster2_impl<V, T, 8>(S, f, x, s); break;
            case 16: launch_cluster2_impl<V, T, 16>(S, f, x, s); break;
            default: launch_cluster2_impl<V, T, 32>(S, f, x, s); break;
        }
        AMGH_LAUNCHED();
        return;
    }
    if (S.staged) {
        switch (S.L) {
            case 1: launch_staged_impl<V, T, 1>(S, f, x, s); break;
            case 2: launch_staged_impl<V, T, 2>(S, f, x, s); break;
            case 4: launch_staged_impl<V, T, 4>(S, f, x, s); break;
            case 8: launch_staged_impl<V, T, 8>(S, f, x, s); break;
            case 16: launch_staged_impl<V, T, 16>(S, f, x, s); break;
            default: launch_staged_impl<V, T, 32>(S, f, x, s); break;
        }
        AMGH_LAUNCHED();
        return;
    }
    switch (S.L) {
        case 1: launch_persistent_impl<V, T, 1>(S, f, x, s); break;
        case 2: launch_persistent_impl<V, T, 2>(S, f, x, s); break;
        case 4: launch_persistent_impl<V, T, 4>(S, f, x, s); break;
        case 8: launch_persistent_impl<V, T, 8>(S, f, x, s); break;
        case 16: launch_persistent_impl<V, T, 16>(S, f, x, s); break;
        default: launch_persistent_impl<V, T, 32>(S, f, x, s); break;
    }
    AMGH_LAUNCHED();
}

bool run_wait_timeout_probe(int* err, cudaStream_t s) {
    DevArray<unsigned> words;
    words.alloc(4);
    words.zero(s);
    AMGH_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    GridBarrier b{words.p, words.p + 1, words.p + 2, err};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(32);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    AMGH_CUDA(cudaLaunchKernelEx(&cfg, wait_timeout_probe_kernel, b));
    AMGH_LAUNCHED();
    int flag = 0;
    AMGH_CUDA(cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGH_CUDA(cudaStreamSynchronize(s));
    return flag != 0;
}

bool cooperative_capture_works() {
    int dev = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return false;
    cudaStream_t s = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    int* d = nullptr;
    int v = 0;
    bool ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&d, sizeof(int)) == cudaSuccess && cudaMemsetAsync(d, 0, sizeof(int), s) == cudaSuccess &&
              cudaStreamSynchronize(s) == cudaSuccess &&
              cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2);
        cfg.blockDim = dim3(32);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const bool launched = cudaLaunchKernelEx(&cfg, coop_probe_kernel, d) == cudaSuccess;
        ok = cudaStreamEndCapture(s, &g) == cudaSuccess && launched && g &&
             cudaGraphInstantiate(&ge, g, 0) == cudaSuccess && cudaGraphLaunch(ge, s) == cudaSuccess &&
             cudaMemcpyAsync(&v, d, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
             cudaStreamSynchronize(s) == cudaSuccess && v == 1;
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (d) cudaFree(d);
    if (s) cudaStreamDestroy(s);
    cudaGetLastError();   // a refused capture leaves a non-sticky error behind
    return ok;
}

template <class V, class T>
int schwarz_staged_cap(const SmootherL<V>& S) {
    const size_t smem = 2 * (size_t)stage_layout(S).stage_bytes();
    switch (S.L) {
        case 1: return staged_cap_impl<V, T, 1>(smem);
        case 2: return staged_cap_impl<V, T, 2>(smem);
        case 4: return staged_cap_impl<V, T, 4>(smem);
        case 8: return staged_cap_impl<V, T, 8>(smem);
        case 16: return staged_cap_impl<V, T, 16>(smem);
        default: return staged_cap_impl<V, T, 32>(smem);
    }
}

template <class V, class T>
int schwarz_persistent_cap(int L) {
    switch (L) {
        case 1: return persistent_cap_impl<V, T, 1>();
        case 2: return persistent_cap_impl<V, T, 2>();
        case 4: return persistent_cap_impl<V, T, 4>();
        case 8: return persistent_cap_impl<V, T, 8>();
        case 16: return persistent_cap_impl<V, T, 16>();
        default: return persistent_cap_impl<V, T, 32>();
    }
}

template <class V, class T, int NBUF>
int stream_cap_nbuf(const SmootherL<V>& S) {
    const size_t smem = stream_smem(S, NBUF);
    switch (S.L) {
        case 1: return stream_cap_impl<V, T, 1, NBUF>(smem);
        case 2: return stream_cap_impl<V, T, 2, NBUF>(smem);
        case 4: return stream_cap_impl<V, T, 4, NBUF>(smem);
        case 8: return stream_cap_impl<V, T, 8, NBUF>(smem);
        case 16: return stream_cap_impl<V, T, 16, NBUF>(smem);
        default: return stream_cap_impl<V, T, 32, NBUF>(smem);
    }
}

template <class V, class T>
bool schwarz_cluster2_ok(const SmootherL<V>& S, int size) {
    if (S.bmax > CL_BMAX) return false;
    switch (S.L) {
        case 1: return cluster2_ok_impl<V, T, 1>(size);
        case 2: return cluster2_ok_impl<V, T, 2>(size);
        case 4: return cluster2_ok_impl<V, T, 4>(size);
        case 8: return cluster2_ok_impl<V, T, 8>(size);
        case 16: return cluster2_ok_impl<V, T, 16>(size);
        default: return cluster2_ok_impl<V, T, 32>(size);
    }
}

template <class V, class T>
bool schwarz_cluster_ok(const SmootherL<V>& S, int size) {
    const size_t smem = 2 * (size_t)stage_layout(S).stage_bytes();
    switch (S.L) {
        case 1: return staged_cluster_ok_impl<V, T, 1>(size, smem);
        case 2: return staged_cluster_ok_impl<V, T, 2>(size, smem);
        case 4: return staged_cluster_ok_impl<V, T, 4>(size, smem);
        case 8: return staged_cluster_ok_impl<V, T, 8>(size, smem);
        case 16: return staged_cluster_ok_impl<V, T, 16>(size, smem);
        default: return staged_cluster_ok_impl<V, T, 32>(size, smem);
    }
}

template <class V, class T>
int schwarz_stream_cap(const SmootherL<V>& S, int nbuf) {
    if (S.bmax > STREAM_BMAX || S.wmax < 1) return 0;
    return nbuf == 1 ? stream_cap_nbuf<V, T, 1>(S) : stream_cap_nbuf<V, T, 2>(S);
}

template <class V, class T>
void launch_schwarz_colourL(const SmootherL<V>& S, int colour, const T* f, T* x, cudaStream_t s) {
    const int cb = S.colour_cta_begin[colour], ce = S.colour_cta_begin[colour + 1];
    if (ce <= cb) return;
    if (S.stream_grid > 0) {
        switch (S.L) {
            case 1: launch_stream_impl<V, T, 1>(S, cb, ce, f, x, s); break;
            case 2: launch_stream_impl<V, T, 2>(S, cb, ce, f, x, s); break;
            case 4: launch_stream_impl<V, T, 4>(S, cb, ce, f, x, s); break;
            case 8: launch_stream_impl<V, T, 8>(S, cb, ce, f, x, s); break;
            case 16: launch_stream_impl<V, T, 16>(S, cb, ce, f, x, s); break;
            default: launch_stream_impl<V, T, 32>(S, cb, ce, f, x, s); break;
        }
        AMGH_LAUNCHED();
        return;
    }
    switch (S.L) {
        case 1: launch_colour_impl<V, T, 1>(S, cb, ce, f, x, s); break;
        case 2: launch_colour_impl<V, T, 2>(S, cb, ce, f, x, s); break;
        case 4: launch_colour_impl<V, T, 4>(S, cb, ce, f, x, s); break;
        case 8: launch_colour_impl<V, T, 8>(S, cb, ce, f, x, s); break;
        case 16: launch_colour_impl<V, T, 16>(S, cb, ce, f, x, s); break;
        default: launch_colour_impl<V, T, 32>(S, cb, ce, f, x, s); break;
    }
    AMGH_LAUNCHED();
}

template <class V, class T>
void launch_schwarz_fused(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s) {
    switch (S.L) {
        case 1: launch_fused_impl<V, T, 1>(S, f, x, s); break;
        case 2: launch_fused_impl<V, T, 2>(S, f, x, s); break;
        case 4: launch_fused_impl<V, T, 4>(S, f, x, s); break;
        case 8: launch_fused_impl<V, T, 8>(S, f, x, s); break;
        case 16: launch_fused_impl<V, T, 16>(S, f, x, s); break;
        default: launch_fused_impl<V, T, 32>(S, f, x, s); break;
    }
    AMGH_LAUNCHED();
}

template <class V>
void launch_slotL_fill(const DevCSR& A, SmootherL<V>& S, cudaStream_t s) {
    if (S.nctas == 0) return;
    slotL_fill_kernel<V><<<S.nctas, CTA_THREADS, 0, s>>>(S.nctas, S.L, S.slot_row.p, A.ptr.p, A.idx.p, A.val.p,
                                                         S.rows.slice_ptr.p, S.rows.col.p, S.rows.val.p);
    AMGH_LAUNCHED();
}

template <class V>
void launch_star_inverseL(const DevCSR& A, int nstars, const int32_t* star_ptr, const int32_t* star_idx,
                          const int32_t* star_cta, const int32_t* star_base, SmootherL<V>& S, int* err_flag,
                          cudaStream_t s) {
    if (nstars == 0) return;
    if (S.bmax <= 8) {
        star_inverse_small_kernel<V><<<(nstars + 7) / 8, 256, 0, s>>>(A.ptr.p, A.idx.p, A.val.p, nstars, star_ptr,
                                                                     star_idx, star_cta, star_base, S.slots, S.bmax,
                                                                     S.inv.p, err_flag);
        AMGH_LAUNCHED();
        return;
    }
    star_inverseL_kernel<V><<<(nstars + 1) / 2, 64, 0, s>>>(A.ptr.p, A.idx.p, A.val.p, nstars, star_ptr, star_idx,
                                                            star_cta, star_base, S.slots, S.bmax, S.inv.p, err_flag);
    AMGH_LAUNCHED();
}

void launch_star_kappa(const DevCSR& A, int nstars, const int32_t* star_ptr, const int32_t* star_idx, double* kappa,
                       int* err_flag, cudaStream_t s) {
    if (nstars == 0) return;
    star_kappa_kernel<<<(nstars + 1) / 2, 64, 0, s>>>(A.ptr.p, A.idx.p, A.val.p, nstars, star_ptr, star_idx,
                                                      reinterpret_cast<unsigned long long*>(kappa), err_flag);
    AMGH_LAUNCHED();
}

#define INST_SCHWARZ(V, T)                                                                                   \
    template void launch_schwarz_colourL<V, T>(const SmootherL<V>&, int, const T*, T*, cudaStream_t);        \
    template void launch_schwarz_fused<V, T>(const SmootherL<V>&, const T*, T*, cudaStream_t);             \
    template void launch_schwarz_persistent<V, T>(const SmootherL<V>&, const T*, T*, cudaStream_t);        \
    template int schwarz_persistent_cap<V, T>(int);                                                      \
    template int schwarz_staged_cap<V, T>(const SmootherL<V>&);                                         \
    template int schwarz_stream_cap<V, T>(const SmootherL<V>&, int);                                    \
    template bool schwarz_cluster_ok<V, T>(const SmootherL<V>&, int);                                   \
    template bool schwarz_cluster2_ok<V, T>(const SmootherL<V>&, int);
INST_SCHWARZ(double, double)
INST_SCHWARZ(float, float)
INST_SCHWARZ(__nv_bfloat16, float)
#define INST_SETUP(V)                                                                                         \
    template void launch_slotL_fill<V>(const DevCSR&, SmootherL<V>&, cudaStream_t);                          \
    template void launch_star_inverseL<V>(const DevCSR&, int, const int32_t*, const int32_t*, const int32_t*, \
                                          const int32_t*, SmootherL<V>&, int*, cudaStream_t);
INST_SETUP(double)
INST_SETUP(float)
INST_SETUP(__nv_bfloat16)

}  // namespace amgh
