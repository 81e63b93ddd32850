// Whole symmetric Schwarz sweep of a small level (the OSS-l1 colour sweep of Section 5) with the
// level's iterate resident in shared memory: one thread-block cluster, every CTA holding a full
// copy of x.  A colour step gathers x from the CTA's own shared memory, and each updated row is
// written to every CTA's copy through distributed shared memory before the hardware cluster
// barrier that ends the step.  The matrix entries, slot metadata, right-hand side and block
// inverse rows of a CTA's next chunk do not depend on x; they are loaded into registers before
// that barrier, so after it only shared-memory gathers, the lane reduction and the block solve
// remain.  The arithmetic and its order are those of the per-colour chunk step.
//
// Work split: the cluster's CTAs each run G chunk groups of 256 threads; group q of the Q = C G
// groups handles chunks cbeg[c] + q, + Q, ... of colour c, so any colour size is covered.  The
// kernel has no spin waits: every thread reaches the same sequence of cluster barriers.
#include <cuda_bf16.h>

#include "schwarz_chunk.cuh"
#include "vcycle_kernels.h"

namespace amgh {

namespace {

constexpr int RS_PREFETCH = 32;   // row-slice entries per lane held in registers (over G groups)
constexpr int RS_BMAX = 16;       // block-inverse entries per row held in registers

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

// one chunk's x-independent data, per thread
template <class V, class T, int PF>
struct ResidentItem {
    int k = -1;   // chunk held, -1: none
    int row = -1, base = 0, bs = 0, w = 0;
    T fr = T(0);
    const int32_t* c = nullptr;
    const V* v = nullptr;
    const V* iv = nullptr;
    int cc[PF];
    V vv[PF];
    T ivr[RS_BMAX];
};

template <class V, class T, int L, int PF>
__device__ __forceinline__ void resident_load(const SmootherLView<V>& S, int k, int gtid, const T* __restrict__ f,
                                              ResidentItem<V, T, PF>& P) {
    constexpr int SLOTS = CTA_THREADS / L;
    const int lane = gtid & 31, slot = gtid / L, sub = gtid % L;
    P.k = k;
    const int64_t gslot = (int64_t)k * SLOTS + slot;
    P.row = S.slot_row[gslot];
    P.base = S.slot_base[gslot];
    P.bs = S.slot_bsize[gslot];
    P.fr = (sub == 0 && P.row >= 0) ? f[P.row] : T(0);
    const int slice = k * WARPS_PER_CTA + (gtid >> 5);
    const int64_t st = S.rows.slice_ptr[slice];
    P.w = (int)((S.rows.slice_ptr[slice + 1] - st) >> 5);
    P.c = S.rows.col + st + lane;
    P.v = S.rows.val + st + lane;
#pragma unroll
    for (int t = 0; t < PF; ++t)
        if (t < P.w) {
            P.cc[t] = P.c[32 * t];
            P.vv[t] = P.v[32 * t];
        }
    P.iv = S.inv + (int64_t)k * S.bmax * SLOTS + slot;
#pragma unroll
    for (int j = 0; j < RS_BMAX; ++j)
        P.ivr[j] = (sub == 0 && P.row >= 0 && j < P.bs) ? widen<T>(P.iv[(int64_t)j * SLOTS]) : T(0);
}

template <class V, class T, int L, int G>
__global__ void __launch_bounds__(G* CTA_THREADS, 1)
    schwarz_resident_kernel(SmootherLView<V> S, int n, const int32_t* __restrict__ sweep, int nsteps,
                            const int32_t* __restrict__ cbeg, const T* __restrict__ f, T* __restrict__ x) {
    constexpr int SLOTS = CTA_THREADS / L;
    constexpr int PF = RS_PREFETCH / G;
    extern __shared__ __align__(16) unsigned char rs_dyn[];
    T* xs = reinterpret_cast<T*>(rs_dyn);
    __shared__ T smem_r[G][CTA_THREADS];
    const unsigned rank = rs_cluster_rank(), C = rs_cluster_size();
    const int g = threadIdx.x / CTA_THREADS, gtid = threadIdx.x % CTA_THREADS;
    const int lane = gtid & 31, slot = gtid / L, sub = gtid % L;
    const int q = (int)rank * G + g, Q = (int)C * G;
    for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = x[i];
    ResidentItem<V, T, PF> P;
    {
        const int c0 = sweep[0], k0 = cbeg[c0] + q;
        if (k0 < cbeg[c0 + 1]) resident_load<V, T, L, PF>(S, k0, gtid, f, P);
    }
    // every copy of x is loaded before any CTA writes into another's copy
    rs_cluster_sync();
    for (int st = 0; st < nsteps; ++st) {
        const int c = sweep[st], end = cbeg[c + 1];
        for (int k = cbeg[c] + q; k < end; k += Q) {
            if (P.k != k) resident_load<V, T, L, PF>(S, k, gtid, f, P);
            T s = T(0);
#pragma unroll
            for (int t = 0; t < PF; ++t)
                if (t < P.w) s = fma(widen<T>(P.vv[t]), xs[P.cc[t]], s);
#pragma unroll 4
            for (int t = PF; t < P.w; ++t) s = fma(widen<T>(P.v[32 * t]), xs[P.c[32 * t]], s);
#pragma unroll
            for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (sub == 0) smem_r[g][slot] = P.row >= 0 ? P.fr - s : T(0);
            rs_group_sync<G>(g);
            T xn = T(0);
            if (sub == 0 && P.row >= 0) {
                T d = T(0);
#pragma unroll
                for (int j = 0; j < RS_BMAX; ++j)
                    if (j < P.bs) d = fma(P.ivr[j], smem_r[g][P.base + j], d);
                for (int j = RS_BMAX; j < P.bs; ++j) d = fma(widen<T>(P.iv[(int64_t)j * SLOTS]), smem_r[g][P.base + j], d);
                xn = xs[P.row] + d;
            }
            // the row's L lanes share its new value and write it into the cluster's copies
            xn = __shfl_sync(0xffffffffu, xn, lane - sub);
            if (P.row >= 0)
                for (unsigned r = (unsigned)sub; r < C; r += L) rs_store_remote(&xs[P.row], r, xn);
            rs_group_sync<G>(g);
            // the next chunk of this colour step, if any, is loaded now
            if (k + Q < end) resident_load<V, T, L, PF>(S, k + Q, gtid, f, P);
        }
        if (st + 1 < nsteps) {
            const int cn = sweep[st + 1], kn = cbeg[cn] + q;
            if (kn < cbeg[cn + 1] && P.k != kn) resident_load<V, T, L, PF>(S, kn, gtid, f, P);
        }
        rs_cluster_sync();
    }
    // after the last barrier every copy is final and no remote store is in flight
    for (int i = (int)rank * blockDim.x + threadIdx.x; i < n; i += (int)C * blockDim.x) x[i] = xs[i];
}

template <class V, class T, int L, int G>
cudaLaunchConfig_t resident_config(int size, int n, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)size);
    cfg.blockDim = dim3(G * CTA_THREADS);
    cfg.dynamicSmemBytes = (size_t)n * sizeof(T);
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <class V, class T, int L, int G>
void launch_resident_impl(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = resident_config<V, T, L, G>(S.resident, S.n, attr);
    cfg.stream = s;
    AMGH_CUDA(cudaLaunchKernelEx(&cfg, schwarz_resident_kernel<V, T, L, G>, view(S), S.n,
                                 (const int32_t*)S.sweep_d.p, (int)S.sweep_d.n,
                                 (const int32_t*)S.colour_cta_begin_d.p, f, x));
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
    auto kern = schwarz_resident_kernel<V, T, L, G>;
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
    cudaLaunchConfig_t cfg = resident_config<V, T, L, G>(size, n, attr);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters >= 1;
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
void launch_resident_g(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s) {
    switch (S.L) {
        case 4: launch_resident_impl<V, T, 4, G>(S, f, x, s); break;
        case 8: launch_resident_impl<V, T, 8, G>(S, f, x, s); break;
        case 16: launch_resident_impl<V, T, 16, G>(S, f, x, s); break;
        case 32: launch_resident_impl<V, T, 32, G>(S, f, x, s); break;
        default: throw CudaError{cudaErrorInvalidConfiguration, "resident sweep needs 4, 8, 16 or 32 lanes per row"};
    }
}

}  // namespace

template <class V, class T>
bool schwarz_resident_ok(const SmootherL<V>& S, int size, int groups) {
    if (S.ncolours < 1 || S.n < 1) return false;
    return groups == 2 ? resident_ok_g<V, T, 2>(S, size) : groups == 1 ? resident_ok_g<V, T, 1>(S, size) : false;
}

template <class V, class T>
void launch_schwarz_resident(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s) {
    if (S.resident_g == 2) launch_resident_g<V, T, 2>(S, f, x, s);
    else launch_resident_g<V, T, 1>(S, f, x, s);
    AMGH_LAUNCHED();
}

#define INST_RESIDENT(V, T)                                                                      \
    template bool schwarz_resident_ok<V, T>(const SmootherL<V>&, int, int);                     \
    template void launch_schwarz_resident<V, T>(const SmootherL<V>&, const T*, T*, cudaStream_t);
INST_RESIDENT(double, double)
INST_RESIDENT(float, float)
INST_RESIDENT(__nv_bfloat16, float)

}  // namespace amgh
