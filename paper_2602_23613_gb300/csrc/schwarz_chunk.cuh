// The per-chunk step of the multiplicative Schwarz smoother (the OSS-l1 colour step of Section 5)
// and the per-colour kernel that applies it, kept in their own file: the finest level's colour
// step is the kernel whose DRAM traffic the benchmark quotes, keyed by this file's contents.
#pragma once
#include <cuda_bf16.h>

#include "layout.h"

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
    // the residual f_i - sum_j a_ij x_j as one FMA chain started at f_i (the row's first lane
    // carries f_i; the lanes' partial sums meet below), and the block update x_i + sum_k
    // (A_BB^-1)_ik r_k as one chain started at x_i: no separate subtraction or addition
    T s = (sub == 0 && row >= 0) ? f[row] : T(0);
#pragma unroll 8
    for (int t = 0; t < w; ++t) s = fma(-widen<T>(v[32 * t]), x[c[32 * t]], s);
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (sub == 0) smem_r[slot] = row >= 0 ? s : T(0);
    __syncthreads();
    if (sub == 0 && row >= 0) {
        const int base = S.slot_base[gslot], bs = S.slot_bsize[gslot];
        const V* iv = S.inv + (int64_t)cta * S.bmax * SLOTS + slot;
        T d = x[row];
        for (int k = 0; k < bs; ++k) d = fma(widen<T>(iv[(int64_t)k * SLOTS]), smem_r[base + k], d);
        x[row] = d;
    }
    __syncthreads();
}

// at most 40 registers per thread: six CTAs per SM, so a colour of the finest level (about 780
// chunks) fits in one wave
template <class V, class T, int L>
__global__ void __launch_bounds__(CTA_THREADS, 6) schwarz_cta_kernel(SmootherLView<V> S, int cta_begin, const T* f, T* x) {
    __shared__ T smem_r[CTA_THREADS];
    schwarz_chunk<V, T, L>(S, cta_begin + blockIdx.x, f, x, smem_r);
}

}  // namespace
}  // namespace amgh
