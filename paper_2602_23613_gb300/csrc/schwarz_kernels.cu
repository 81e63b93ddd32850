// Multiplicative Schwarz on node stars (the OSS-l1 smoother of Section 5): one colour per launch
// over CTA chunks, or a whole symmetric sweep of a small level in one single-CTA launch; plus the
// setup of the chunk layout (slot rows, star-block inverses, conditioning estimate).
#include <cuda_bf16.h>

#include <type_traits>

#include "star_invert.cuh"
#include "vcycle_kernels.h"

namespace amgh {

namespace {

template <class T, class V> __device__ __forceinline__ T widen(V v) { return (T)v; }
template <> __device__ __forceinline__ float widen<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ double widen<double, __nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <class V> __device__ __forceinline__ V narrow(double x);
template <> __device__ __forceinline__ double narrow<double>(double x) { return x; }
template <> __device__ __forceinline__ float narrow<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ __nv_bfloat16 narrow<__nv_bfloat16>(double x) { return __float2bfloat16_rn((float)x); }

// One chunk (CTA) of one colour: every row slot (L lanes) forms f_i - (A x)_i for its row, the
// star's residuals meet in shared memory, and each row applies its row of A_BB^{-1}:
// x_B += A_BB^{-1} r_B.  Stars of one colour share no row and no coupling, so chunks of a colour
// are independent.  All threads of the CTA call this (it holds two barriers).
template <class V, class T, int L>
__device__ __forceinline__ void schwarz_chunk(const SmootherLView<V>& S, int cta, const T* f, T* x, T* smem_r) {
    constexpr int SLOTS = CTA_THREADS / L;
    const int tid = threadIdx.x, lane = tid & 31, slot = tid / L, sub = tid % L;
    const int64_t gslot = (int64_t)cta * SLOTS + slot;
    const int row = S.slot_row[gslot];
    const int slice = cta * WARPS_PER_CTA + (tid >> 5);
    const int64_t st = S.rows.slice_ptr[slice];
    const int w = (int)((S.rows.slice_ptr[slice + 1] - st) >> 5);
    const int32_t* c = S.rows.col + st + lane;
    const V* v = S.rows.val + st + lane;
    T s = T(0);
#pragma unroll 4
    for (int t = 0; t < w; ++t) s = fma(widen<T>(v[32 * t]), x[c[32 * t]], s);
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (sub == 0) smem_r[slot] = row >= 0 ? f[row] - s : T(0);
    __syncthreads();
    if (sub == 0 && row >= 0) {
        const int base = S.slot_base[gslot], bs = S.slot_bsize[gslot];
        const V* iv = S.inv + (int64_t)cta * S.bmax * SLOTS + slot;
        T d = T(0);
        for (int k = 0; k < bs; ++k) d = fma(widen<T>(iv[(int64_t)k * SLOTS]), smem_r[base + k], d);
        x[row] += d;
    }
    __syncthreads();
}

template <class V, class T, int L>
__global__ void __launch_bounds__(CTA_THREADS) schwarz_cta_kernel(SmootherLView<V> S, int cta_begin, const T* f, T* x) {
    __shared__ T smem_r[CTA_THREADS];
    schwarz_chunk<V, T, L>(S, cta_begin + blockIdx.x, f, x, smem_r);
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
    schwarz_cta_kernel<V, T, L><<<ce - cb, CTA_THREADS, 0, s>>>(view(S), cb, f, x);
}

template <class V, class T, int L>
void launch_fused_impl(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s) {
    schwarz_fused_kernel<V, T, L><<<1, CTA_THREADS, 0, s>>>(view(S), S.sweep_d.p, (int)S.sweep_d.n,
                                                             S.colour_cta_begin_d.p, f, x);
}

}  // namespace

template <class V, class T>
void launch_schwarz_colourL(const SmootherL<V>& S, int colour, const T* f, T* x, cudaStream_t s) {
    const int cb = S.colour_cta_begin[colour], ce = S.colour_cta_begin[colour + 1];
    if (ce <= cb) return;
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
    template void launch_schwarz_fused<V, T>(const SmootherL<V>&, const T*, T*, cudaStream_t);
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
