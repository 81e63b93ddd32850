// Sliced-ELL passes with L lanes per row (residual, l1-Jacobi, restriction, prolongation) and the
// setup fill of the layout.  L = 1 is the finest-level form: every thread owns a row and only
// multiplies and adds (no reduction instructions on the scarce FP64 pipe).  Larger L spread the
// long rows of coarse Galerkin operators over several lanes; the partial sums of a row are then
// combined by xor-shuffles inside the L-lane group.
#include <cuda_bf16.h>

#include <type_traits>

#include "vcycle_kernels.h"

namespace amgh {

namespace {

template <class V> __device__ __forceinline__ double to_d(V v) { return (double)v; }
template <> __device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <class V> __device__ __forceinline__ float to_f(V v) { return (float)v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class A, class V> __device__ __forceinline__ A widen(V v) {
    if constexpr (std::is_same<A, double>::value) return to_d<V>(v);
    else return to_f<V>(v);
}

template <class V> __device__ __forceinline__ V narrow(double x);
template <> __device__ __forceinline__ double narrow<double>(double x) { return x; }
template <> __device__ __forceinline__ float narrow<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ __nv_bfloat16 narrow<__nv_bfloat16>(double x) { return __float2bfloat16_rn((float)x); }

template <class V, class TX, class TY, int MODE, int L>
__global__ void __launch_bounds__(256) sellL_kernel(SellLView<V> M, const TX* __restrict__ x, const TY* __restrict__ f,
                                                    const TY* __restrict__ dinv, TY* __restrict__ y) {
    using Acc = typename std::conditional<std::is_same<TX, double>::value || std::is_same<TY, double>::value,
                                          double, float>::type;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = gt >> 5, lane = threadIdx.x & 31;
    if (slice >= M.nslices) return;                      // uniform over the warp
    const int row = slice * (32 / L) + lane / L;
    const int64_t st = M.slice_ptr[slice];
    const int w = (int)((M.slice_ptr[slice + 1] - st) >> 5);
    const int32_t* __restrict__ c = M.col + st + lane;
    const V* __restrict__ v = M.val + st + lane;
    Acc s = Acc(0);
#pragma unroll 4
    for (int t = 0; t < w; ++t) s = fma(widen<Acc>(v[32 * t]), (Acc)x[c[32 * t]], s);
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((lane % L) != 0 || row >= M.nrows) return;
    if (MODE == SM_AX) y[row] = (TY)s;
    else if (MODE == SM_RESID) y[row] = (TY)((Acc)f[row] - s);
    else if (MODE == SM_L1) y[row] = (TY)((Acc)x[row] + (Acc)dinv[row] * ((Acc)f[row] - s));
    else y[row] = (TY)((Acc)y[row] + s);
}

template <class V, class TX, class TY, int MODE>
void launch_mode(int L, const SellL<V>& M, const TX* x, const TY* f, const TY* dinv, TY* y, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (int)(((int64_t)M.nslices * 32 + threads - 1) / threads);
    auto v = view(M);
    switch (L) {
        case 1: sellL_kernel<V, TX, TY, MODE, 1><<<blocks, threads, 0, s>>>(v, x, f, dinv, y); break;
        case 2: sellL_kernel<V, TX, TY, MODE, 2><<<blocks, threads, 0, s>>>(v, x, f, dinv, y); break;
        case 4: sellL_kernel<V, TX, TY, MODE, 4><<<blocks, threads, 0, s>>>(v, x, f, dinv, y); break;
        case 8: sellL_kernel<V, TX, TY, MODE, 8><<<blocks, threads, 0, s>>>(v, x, f, dinv, y); break;
        case 16: sellL_kernel<V, TX, TY, MODE, 16><<<blocks, threads, 0, s>>>(v, x, f, dinv, y); break;
        default: sellL_kernel<V, TX, TY, MODE, 32><<<blocks, threads, 0, s>>>(v, x, f, dinv, y); break;
    }
    AMGH_LAUNCHED();
}

// Fused residual and restriction, r_c = P^T (f - A y), written by associativity as
// P^T f - W y with W = P^T A formed at setup: one row-gather pass over the rows of P^T and W, no
// fine residual written anywhere and no atomics.  PT and W have the same rows and the same L, so
// one lane group owns row c in both.
template <class V, class TX, class TY, int L>
__global__ void __launch_bounds__(256) rr_kernel(SellLView<V> PT, SellLView<V> W, const TX* __restrict__ f,
                                                 const TX* __restrict__ y, TY* __restrict__ out) {
    using Acc = typename std::conditional<std::is_same<TX, double>::value || std::is_same<TY, double>::value,
                                          double, float>::type;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = gt >> 5, lane = threadIdx.x & 31;
    if (slice >= PT.nslices) return;                     // uniform over the warp
    const int row = slice * (32 / L) + lane / L;
    Acc s = Acc(0);
    {
        const int64_t st = PT.slice_ptr[slice];
        const int w = (int)((PT.slice_ptr[slice + 1] - st) >> 5);
        const int32_t* __restrict__ c = PT.col + st + lane;
        const V* __restrict__ v = PT.val + st + lane;
#pragma unroll 4
        for (int t = 0; t < w; ++t) s = fma(widen<Acc>(v[32 * t]), (Acc)f[c[32 * t]], s);
    }
    {
        const int64_t st = W.slice_ptr[slice];
        const int w = (int)((W.slice_ptr[slice + 1] - st) >> 5);
        const int32_t* __restrict__ c = W.col + st + lane;
        const V* __restrict__ v = W.val + st + lane;
#pragma unroll 4
        for (int t = 0; t < w; ++t) s = fma(-widen<Acc>(v[32 * t]), (Acc)y[c[32 * t]], s);
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((lane % L) != 0 || row >= PT.nrows) return;
    out[row] = (TY)s;
}

template <class V>
__global__ void sellL_fill_kernel(int n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                  const double* __restrict__ val, int nslices, int L,
                                  const int64_t* __restrict__ sptr, int32_t* __restrict__ scol, V* __restrict__ sval) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = gt >> 5, lane = gt & 31;
    if (slice >= nslices) return;
    const int row = slice * (32 / L) + lane / L, sub = lane % L;
    const int64_t st = sptr[slice];
    const int w = (int)((sptr[slice + 1] - st) >> 5);
    int b = 0, len = 0;
    if (row < n) { b = ptr[row]; len = ptr[row + 1] - b; }
    const int pad_col = len > 0 ? idx[b + len - 1] : 0;
    for (int t = 0; t < w; ++t) {
        const int e = t * L + sub;
        const int64_t o = st + 32 * (int64_t)t + lane;
        if (e < len) { scol[o] = idx[b + e]; sval[o] = narrow<V>(val[b + e]); }
        else { scol[o] = pad_col; sval[o] = narrow<V>(0.0); }
    }
}

}  // namespace

template <class V, class TX, class TY>
void launch_sellL(int mode, const SellL<V>& M, const TX* x, const TY* f, const TY* dinv, TY* y, cudaStream_t s) {
    if (M.nslices == 0) return;
    switch (mode) {
        case SM_AX: launch_mode<V, TX, TY, SM_AX>(M.L, M, x, f, dinv, y, s); break;
        case SM_ADD: launch_mode<V, TX, TY, SM_ADD>(M.L, M, x, f, dinv, y, s); break;
        case SM_RESID:
            if constexpr (std::is_same<TX, TY>::value) launch_mode<V, TX, TY, SM_RESID>(M.L, M, x, f, dinv, y, s);
            break;
        default:
            if constexpr (std::is_same<TX, TY>::value) launch_mode<V, TX, TY, SM_L1>(M.L, M, x, f, dinv, y, s);
            break;
    }
}

template <class V, class TX, class TY>
void launch_rr(const SellL<V>& PT, const SellL<V>& W, const TX* f, const TX* y, TY* out, cudaStream_t s) {
    if (PT.nslices == 0) return;
    if (W.nslices != PT.nslices || W.L != PT.L || W.nrows != PT.nrows)
        throw CudaError{cudaErrorInvalidValue, "launch_rr: P^T and W layouts differ"};
    const int threads = 256;
    const int blocks = (int)(((int64_t)PT.nslices * 32 + threads - 1) / threads);
    auto a = view(PT);
    auto b = view(W);
    switch (PT.L) {
        case 1: rr_kernel<V, TX, TY, 1><<<blocks, threads, 0, s>>>(a, b, f, y, out); break;
        case 2: rr_kernel<V, TX, TY, 2><<<blocks, threads, 0, s>>>(a, b, f, y, out); break;
        case 4: rr_kernel<V, TX, TY, 4><<<blocks, threads, 0, s>>>(a, b, f, y, out); break;
        case 8: rr_kernel<V, TX, TY, 8><<<blocks, threads, 0, s>>>(a, b, f, y, out); break;
        case 16: rr_kernel<V, TX, TY, 16><<<blocks, threads, 0, s>>>(a, b, f, y, out); break;
        default: rr_kernel<V, TX, TY, 32><<<blocks, threads, 0, s>>>(a, b, f, y, out); break;
    }
    AMGH_LAUNCHED();
}

template <class V>
void launch_sellL_fill(const DevCSR& M, SellL<V>& S, cudaStream_t s) {
    if (S.nslices == 0) return;
    const int blocks = (int)(((int64_t)S.nslices * 32 + 255) / 256);
    sellL_fill_kernel<V><<<blocks, 256, 0, s>>>(M.nrows, M.ptr.p, M.idx.p, M.val.p, S.nslices, S.L, S.slice_ptr.p,
                                                S.col.p, S.val.p);
    AMGH_LAUNCHED();
}

#define INST_SELL(V, TX, TY) \
    template void launch_sellL<V, TX, TY>(int, const SellL<V>&, const TX*, const TY*, const TY*, TY*, cudaStream_t);
INST_SELL(double, double, double)
INST_SELL(double, double, float)
INST_SELL(double, float, double)
INST_SELL(double, float, float)
INST_SELL(float, float, float)
INST_SELL(float, float, double)
INST_SELL(float, double, float)
INST_SELL(float, double, double)
INST_SELL(__nv_bfloat16, float, float)
INST_SELL(__nv_bfloat16, float, double)
INST_SELL(__nv_bfloat16, double, float)
INST_SELL(__nv_bfloat16, double, double)
#define INST_RR(V, TX, TY) \
    template void launch_rr<V, TX, TY>(const SellL<V>&, const SellL<V>&, const TX*, const TX*, TY*, cudaStream_t);
INST_RR(double, double, double)
INST_RR(double, double, float)
INST_RR(float, double, double)
INST_RR(float, double, float)
INST_RR(float, float, float)
INST_RR(float, float, double)
INST_RR(__nv_bfloat16, double, double)
INST_RR(__nv_bfloat16, double, float)
INST_RR(__nv_bfloat16, float, float)
INST_RR(__nv_bfloat16, float, double)
template void launch_sellL_fill<double>(const DevCSR&, SellL<double>&, cudaStream_t);
template void launch_sellL_fill<float>(const DevCSR&, SellL<float>&, cudaStream_t);
template void launch_sellL_fill<__nv_bfloat16>(const DevCSR&, SellL<__nv_bfloat16>&, cudaStream_t);

}  // namespace amgh
