// Whole symmetric Schwarz sweep of a small level (the OSS-l1 colour sweep of Section 5) with the
// level's iterate resident in shared memory: one thread-block cluster, every CTA holding a full
// copy of x.  A colour step gathers x from the CTA's own shared memory, and each updated row is
// written to every CTA's copy through distributed shared memory before the hardware cluster
// barrier that ends the step.  The matrix entries, slot metadata, right-hand side and block
// inverse rows of a CTA's next chunk do not depend on x; they are loaded into registers before
// that barrier, so after it only shared-memory gathers, the lane reduction and the block solve
// remain.
//
// Work split: the cluster's CTAs each run G chunk groups of 256 threads; the j-th chunk of a
// colour step goes to group j mod Q of the Q = C G groups (group q = g C + rank, so a step's
// first C chunks land on C different SMs), so any colour size is covered.  Each group walks its
// own host-built list of (step, chunk) items through a software pipeline: the id of the item
// three ahead, the slot metadata of the item two ahead, and the matrix entries, block-inverse
// row and right-hand side of the next item are loaded while the current one computes.  The
// residual of a lane's entries is summed in two interleaved partial sums (even and odd entries)
// to keep two FP64 FMA chains in flight.  In this form the kernel has no spin waits: every thread
// reaches the same sequence of cluster barriers.
//
// The same kernel body also runs as a cooperative grid of any size (GRID = true, launch mode 9):
// x stays in global memory, updated rows are stored there, and the colour steps are ordered by a
// counter barrier whose polls are bounded (a poll that gives up raises the abort word and the
// handle's wait flag, and every CTA returns).
#include <cuda_bf16.h>

#include <climits>
#include <vector>

#include "schwarz_chunk.cuh"
#include "vcycle_kernels.h"

namespace amgh {

namespace {

constexpr int RS_PREFETCH = 32;   // row-slice entries per lane held in registers (over G groups)
constexpr int RS_BMAX = 16;       // block-inverse entries per row held in registers (over G groups)

__device__ __forceinline__ void rs_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned rs_cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned rs_cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

template <int G>
__device__ __forceinline__ void rs_group_sync(int g) {
    if (G == 1) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(CTA_THREADS) : "memory");
    }
}

// store v at the same shared-memory offset as `local` in CTA `rank` of the cluster
__device__ __forceinline__ void rs_store_remote(double* local, unsigned rank, double v) {
    uint32_t a = (uint32_t)__cvta_generic_to_shared(local), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(v) : "memory");
}
__device__ __forceinline__ void rs_store_remote(float* local, unsigned rank, float v) {
    uint32_t a = (uint32_t)__cvta_generic_to_shared(local), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
}

// Where the x-independent data of one item (a chunk of a colour step) lives, per thread: its
// slot's row, star base and size, and its warp's slice.  The loads are issued one item before
// they are used and only read at that point, so no round trip waits in between.
struct RsMeta {
    int step = INT_MAX;   // colour step of the item; INT_MAX: none
    int k = 0, row = -1, base = 0, bs = 0;
    int64_t s0 = 0, s1 = 0;   // slice bounds (entries)
};

template <class V, int L>
__device__ __forceinline__ void rs_meta(const SmootherLView<V>& S, int2 id, int gtid, RsMeta& m) {
    constexpr int SLOTS = CTA_THREADS / L;
    m.step = id.x;
    m.k = id.y;
    m.row = -1;
    m.bs = 0;
    m.s0 = m.s1 = 0;
    if (id.x == INT_MAX) return;
    const int64_t gslot = (int64_t)id.y * SLOTS + gtid / L;
    m.row = S.slot_row[gslot];
    m.base = S.slot_base[gslot];
    m.bs = S.slot_bsize[gslot];
    const int slice = id.y * WARPS_PER_CTA + (gtid >> 5);
    m.s0 = S.rows.slice_ptr[slice];
    m.s1 = S.rows.slice_ptr[slice + 1];
}

__device__ __forceinline__ int2 rs_id(const int2* __restrict__ items, int i, int i1) {
    return i < i1 ? items[i] : make_int2(INT_MAX, 0);
}

// Grid-wide barrier of the pipelined sweep: each CTA adds one to a counter (zeroed before the
// launch) with release semantics and thread 0 polls it with acquire loads until all CTAs of
// barrier `round` have arrived.  The wait is bounded: after SPIN_LIMIT polls it raises the abort
// word and the error flag; a CTA that sees the abort word (read every 16th poll) gives up too.
// False when it gave up.
constexpr long long RS_SPIN_LIMIT = 1ll << 20;

__device__ __forceinline__ unsigned rs_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool rs_grid_sync(const GridBarrier& b, unsigned round) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(b.count) : "memory");
        const unsigned target = round * gridDim.x;
        long long it = 0;
        while (rs_ld_acquire(b.count) < target) {
            // the abort word is read on every 16th poll only, so the poll loop issues one load
            if ((++it & 15) == 0 && (rs_ld_acquire(b.abort) != 0u || it > RS_SPIN_LIMIT)) {
                atomicExch(b.abort, 1u);
                atomicExch(b.err, 1);
                good = 0;
                break;
            }
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// GRID = false: the resident sweep (one cluster, x in every CTA's shared memory, hardware cluster
// barrier).  GRID = true: the same pipelined item walk over a cooperative grid of any size, with x
// in global memory (gathers from L2) and the counter barrier above, so the FP64 work of a step
// spreads over as many SMs as the grid has CTAs.
template <class V, class T, int L, int G, bool GRID>
__global__ void __launch_bounds__(G* CTA_THREADS, 1)
    schwarz_resident_kernel(SmootherLView<V> S, int n, const int2* __restrict__ items, const int32_t* __restrict__ iptr,
                            int nsteps, const T* __restrict__ f, T* __restrict__ x, GridBarrier bar) {
    constexpr int SLOTS = CTA_THREADS / L;
    constexpr int PF = RS_PREFETCH / G;
    constexpr int BM = RS_BMAX / G;
    extern __shared__ __align__(16) unsigned char rs_dyn[];
    T* xs = GRID ? x : reinterpret_cast<T*>(rs_dyn);
    __shared__ T smem_r[G][CTA_THREADS];
    const unsigned rank = GRID ? blockIdx.x : rs_cluster_rank(), C = GRID ? gridDim.x : rs_cluster_size();
    const int g = threadIdx.x / CTA_THREADS, gtid = threadIdx.x % CTA_THREADS;
    const int lane = gtid & 31, slot = gtid / L, sub = gtid % L;
    // group-major: the first C chunks of a colour step go to C different CTAs
    const int q = g * (int)C + (int)rank;
    const int i1 = iptr[q + 1];
    int i = iptr[q];
    if (!GRID)
        for (int j = threadIdx.x; j < n; j += blockDim.x) xs[j] = x[j];

    // pipeline: entries of item i (registers), metadata of items i and i+1, id of item i+2
    RsMeta mc, mn;
    rs_meta<V, L>(S, rs_id(items, i, i1), gtid, mc);
    rs_meta<V, L>(S, rs_id(items, i + 1, i1), gtid, mn);
    int2 id2 = rs_id(items, i + 2, i1);
    int cc[PF];
    V vv[PF];
    T ivr[BM];
    T fr = T(0);
    {
        const int w = (int)((mc.s1 - mc.s0) >> 5);
        const int32_t* cp = S.rows.col + mc.s0 + lane;
        const V* vp = S.rows.val + mc.s0 + lane;
#pragma unroll
        for (int t = 0; t < PF; ++t)
            if (t < w) {
                cc[t] = cp[32 * t];
                vv[t] = vp[32 * t];
            }
        const V* iv = S.inv + (int64_t)mc.k * S.bmax * SLOTS + slot;
        const bool own = sub == 0 && mc.row >= 0;
#pragma unroll
        for (int j = 0; j < BM; ++j) ivr[j] = (own && j < mc.bs) ? widen<T>(iv[(int64_t)j * SLOTS]) : T(0);
        fr = own ? f[mc.row] : T(0);
    }
    // every copy of x is loaded before any CTA writes into another's copy
    if (!GRID) rs_cluster_sync();
    for (int st = 0; st < nsteps; ++st) {
        while (mc.step == st) {
            // metadata two items ahead, id three items ahead
            RsMeta m2;
            rs_meta<V, L>(S, id2, gtid, m2);
            const int2 id3 = rs_id(items, i + 3, i1);
            const int w = (int)((mc.s1 - mc.s0) >> 5);
            const int wn = (int)((mn.s1 - mn.s0) >> 5);
            const int32_t* cpn = S.rows.col + mn.s0 + lane;
            const V* vpn = S.rows.val + mn.s0 + lane;
            // residual of the current item, started at f_i on the row's first lane; each
            // register is refilled with the next item's entry as soon as it has been used
            T s0 = fr, s1 = T(0);
#pragma unroll
            for (int t = 0; t < PF; ++t) {
                if (t < w) {
                    if (t & 1) s1 = fma(-widen<T>(vv[t]), xs[cc[t]], s1);
                    else s0 = fma(-widen<T>(vv[t]), xs[cc[t]], s0);
                }
                if (t < wn) {
                    cc[t] = cpn[32 * t];
                    vv[t] = vpn[32 * t];
                }
            }
            {
                const int32_t* cp = S.rows.col + mc.s0 + lane;
                const V* vp = S.rows.val + mc.s0 + lane;
                for (int t = PF; t < w; ++t) {
                    if (t & 1) s1 = fma(-widen<T>(vp[32 * t]), xs[cp[32 * t]], s1);
                    else s0 = fma(-widen<T>(vp[32 * t]), xs[cp[32 * t]], s0);
                }
            }
            T s = s0 + s1;
#pragma unroll
            for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (sub == 0) smem_r[g][slot] = mc.row >= 0 ? s : T(0);
            rs_group_sync<G>(g);
            T xn = T(0);
            if (sub == 0 && mc.row >= 0) {
                // the block update as one chain started at x_i
                T d = xs[mc.row];
#pragma unroll
                for (int j = 0; j < BM; ++j)
                    if (j < mc.bs) d = fma(ivr[j], smem_r[g][mc.base + j], d);
                const V* iv = S.inv + (int64_t)mc.k * S.bmax * SLOTS + slot;
                for (int j = BM; j < mc.bs; ++j) d = fma(widen<T>(iv[(int64_t)j * SLOTS]), smem_r[g][mc.base + j], d);
                xn = d;
            }
            if (GRID) {
                if (sub == 0 && mc.row >= 0) x[mc.row] = xn;
            } else {
                // the row's L lanes share its new value and write it into the cluster's copies
                xn = __shfl_sync(0xffffffffu, xn, lane - sub);
                if (mc.row >= 0)
                    for (unsigned r = (unsigned)sub; r < C; r += L) rs_store_remote(&xs[mc.row], r, xn);
            }
            // block-inverse row and right-hand side of the next item
            {
                const V* iv = S.inv + (int64_t)mn.k * S.bmax * SLOTS + slot;
                const bool own = sub == 0 && mn.row >= 0;
#pragma unroll
                for (int j = 0; j < BM; ++j) ivr[j] = (own && j < mn.bs) ? widen<T>(iv[(int64_t)j * SLOTS]) : T(0);
                fr = own ? f[mn.row] : T(0);
            }
            rs_group_sync<G>(g);
            mc = mn;
            mn = m2;
            id2 = id3;
            ++i;
        }
        if (GRID) {
            if (st + 1 < nsteps && !rs_grid_sync(bar, (unsigned)st + 1u)) return;
        } else {
            rs_cluster_sync();
        }
    }
    if (GRID) return;
    // after the last barrier every copy is final and no remote store is in flight
    for (int j = (int)rank * blockDim.x + threadIdx.x; j < n; j += (int)C * blockDim.x) x[j] = xs[j];
}

template <class V, class T, int L, int G, bool GRID>
cudaLaunchConfig_t resident_config(int size, int n, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)size);
    cfg.blockDim = dim3(G * CTA_THREADS);
    cfg.dynamicSmemBytes = GRID ? 0 : (size_t)n * sizeof(T);
    if (GRID) {
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
    } else {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)size;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <class V, class T, int L, int G, bool GRID>
void launch_resident_impl(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s) {
    if (S.rs_size != S.resident || S.rs_groups != G)
        throw CudaError{cudaErrorInvalidConfiguration, "resident sweep launched without its item lists"};
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = resident_config<V, T, L, G, GRID>(S.resident, S.n, attr);
    cfg.stream = s;
    // the grid barrier counts arrivals from zero in every launch
    if (GRID) AMGH_CUDA(cudaMemsetAsync(S.bar.p, 0, sizeof(unsigned), s));
    AMGH_CUDA(cudaLaunchKernelEx(&cfg, schwarz_resident_kernel<V, T, L, G, GRID>, view(S), S.n,
                                 reinterpret_cast<const int2*>(S.rs_items.p), (const int32_t*)S.rs_ptr.p,
                                 (int)S.sweep_d.n, f, x, S.barrier()));
}

// raises the kernel's shared-memory and cluster-size limits, then asks whether one cluster fits
template <class V, class T, int L, int G>
bool resident_ok_impl(int size, int n) {
    if (size < 1 || size > 16 || n < 1) return false;
    int dev = 0, maxsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    auto kern = schwarz_resident_kernel<V, T, L, G, false>;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    // the limit is per kernel, not per level: always the device's whole opt-in budget
    const int cap = maxsm - (int)fa.sharedSizeBytes;
    const size_t smem = (size_t)n * sizeof(T);
    if (cap <= 0 || smem > (size_t)cap) return false;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) != cudaSuccess ||
        (size > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = resident_config<V, T, L, G, false>(size, n, attr);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters >= 1;
}

// co-resident CTAs of the pipelined grid sweep on this device
template <class V, class T, int L, int G>
int pipeline_cap_impl() {
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, schwarz_resident_kernel<V, T, L, G, true>,
                                                      G * CTA_THREADS, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nsm * per_sm;
}

template <class V, class T, int G>
bool resident_ok_g(const SmootherL<V>& S, int size) {
    switch (S.L) {
        case 4: return resident_ok_impl<V, T, 4, G>(size, S.n);
        case 8: return resident_ok_impl<V, T, 8, G>(size, S.n);
        case 16: return resident_ok_impl<V, T, 16, G>(size, S.n);
        case 32: return resident_ok_impl<V, T, 32, G>(size, S.n);
        default: return false;
    }
}

template <class V, class T, int G>
int pipeline_cap_g(const SmootherL<V>& S) {
    switch (S.L) {
        case 4: return pipeline_cap_impl<V, T, 4, G>();
        case 8: return pipeline_cap_impl<V, T, 8, G>();
        case 16: return pipeline_cap_impl<V, T, 16, G>();
        case 32: return pipeline_cap_impl<V, T, 32, G>();
        default: return 0;
    }
}

template <class V, class T, int G, bool GRID>
void launch_resident_g(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s) {
    switch (S.L) {
        case 4: launch_resident_impl<V, T, 4, G, GRID>(S, f, x, s); break;
        case 8: launch_resident_impl<V, T, 8, G, GRID>(S, f, x, s); break;
        case 16: launch_resident_impl<V, T, 16, G, GRID>(S, f, x, s); break;
        case 32: launch_resident_impl<V, T, 32, G, GRID>(S, f, x, s); break;
        default: throw CudaError{cudaErrorInvalidConfiguration, "resident sweep needs 4, 8, 16 or 32 lanes per row"};
    }
}

}  // namespace

template <class V, class T>
bool schwarz_resident_ok(const SmootherL<V>& S, int size, int groups) {
    if (S.ncolours < 1 || S.n < 1) return false;
    return groups == 2 ? resident_ok_g<V, T, 2>(S, size) : groups == 1 ? resident_ok_g<V, T, 1>(S, size) : false;
}

template <class V>
void schwarz_resident_prepare(SmootherL<V>& S, int size, int groups, cudaStream_t s) {
    if (S.rs_size == size && S.rs_groups == groups) return;
    const int Q = size * groups, C = S.ncolours;
    std::vector<std::vector<int32_t>> per(Q);
    int st = 0;
    auto add = [&](int c) {
        for (int k = S.colour_cta_begin[c], j = 0; k < S.colour_cta_begin[c + 1]; ++k, ++j) {
            per[j % Q].push_back(st);
            per[j % Q].push_back(k);
        }
        ++st;
    };
    for (int c = 0; c < C; ++c) add(c);
    for (int c = C - 2; c >= 0; --c) add(c);
    std::vector<int32_t> items, ptr(Q + 1, 0);
    for (int q = 0; q < Q; ++q) {
        items.insert(items.end(), per[q].begin(), per[q].end());
        ptr[q + 1] = (int32_t)(items.size() / 2);
    }
    if (items.empty()) items.assign(2, 0);   // a valid (unused) address
    S.rs_items.upload(items, s);
    S.rs_ptr.upload(ptr, s);
    S.rs_size = size;
    S.rs_groups = groups;
}

template <class V, class T>
int schwarz_pipeline_cap(const SmootherL<V>& S, int groups) {
    if (S.ncolours < 1 || S.n < 1) return 0;
    return groups == 2 ? pipeline_cap_g<V, T, 2>(S) : groups == 1 ? pipeline_cap_g<V, T, 1>(S) : 0;
}

template <class V, class T>
void launch_schwarz_resident(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s) {
    if (S.resident_grid) {
        if (S.resident_g == 2) launch_resident_g<V, T, 2, true>(S, f, x, s);
        else launch_resident_g<V, T, 1, true>(S, f, x, s);
    } else {
        if (S.resident_g == 2) launch_resident_g<V, T, 2, false>(S, f, x, s);
        else launch_resident_g<V, T, 1, false>(S, f, x, s);
    }
    AMGH_LAUNCHED();
}

#define INST_RESIDENT(V, T)                                                                      \
    template bool schwarz_resident_ok<V, T>(const SmootherL<V>&, int, int);                     \
    template int schwarz_pipeline_cap<V, T>(const SmootherL<V>&, int);                          \
    template void schwarz_resident_prepare<V>(SmootherL<V>&, int, int, cudaStream_t);           \
    template void launch_schwarz_resident<V, T>(const SmootherL<V>&, const T*, T*, cudaStream_t);
INST_RESIDENT(double, double)
INST_RESIDENT(float, float)
INST_RESIDENT(__nv_bfloat16, float)

}  // namespace amgh
