// V-cycle and Krylov kernels.  Every sparse pass is thread-per-row over a 32-row SELL slice:
// each thread accumulates its own row, so no floating-point shuffle reduction is spent (the
// FP64 pipe of this part is the scarce resource, one FMA per 12-byte nonzero already).
#include <cuda_bf16.h>

#include "kernels.h"

namespace amgh {

namespace {

template <class V> __device__ __forceinline__ float to_f(V v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class V, class T> __device__ __forceinline__ T widen(V v);
template <> __device__ __forceinline__ double widen<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float widen<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float widen<__nv_bfloat16, float>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class V, class T>
__device__ __forceinline__ T row_dot(const SellView<V>& A, int64_t st, int w, int lane, const T* __restrict__ x) {
    T s = T(0);
    const int32_t* __restrict__ c = A.col + st + lane;
    const V* __restrict__ v = A.val + st + lane;
#pragma unroll 4
    for (int t = 0; t < w; ++t) s = fma(widen<V, T>(v[32 * t]), x[c[32 * t]], s);
    return s;
}

template <class V, class T, int MODE>
__global__ void __launch_bounds__(256) sell_kernel(SellView<V> A, const T* __restrict__ x, const T* __restrict__ f,
                                                   const T* __restrict__ dinv, T* __restrict__ y) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = row >> 5, lane = row & 31;
    if (slice >= A.nslices) return;
    const int64_t st = A.slice_ptr[slice];
    const int w = (int)((A.slice_ptr[slice + 1] - st) >> 5);
    const T s = row_dot<V, T>(A, st, w, lane, x);
    if (row >= A.nrows) return;
    if (MODE == SELL_AX) y[row] = s;
    else if (MODE == SELL_RESID) y[row] = f[row] - s;
    else if (MODE == SELL_L1) y[row] = x[row] + dinv[row] * (f[row] - s);
    else y[row] += s;
}

// y = inv x for a dense n x n operator (the coarsest inverse or the dense tail): a warp per row,
// lanes over the row (coalesced), shuffle reduction
template <class T>
__global__ void coarse_apply_kernel(const T* __restrict__ inv, int n, const T* __restrict__ x, T* __restrict__ y) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= n) return;
    const T* r = inv + (int64_t)row * n;
    T s = T(0);
    for (int k = lane; k < n; k += 32) s = fma(r[k], x[k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
}

// ---------------- FP64 Krylov vector kernels (fixed grid, deterministic) -----------------------
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[RED_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < RED_THREADS / 32; ++i) t += red[i];
    return t;   // valid in thread 0
}

__global__ void __launch_bounds__(RED_THREADS) spmv_dot_kernel(SellView<double> A, const double* __restrict__ p,
                                                              double* __restrict__ q, double* __restrict__ partial) {
    double acc = 0.0;
    const int nrows_pad = A.nslices * 32;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < nrows_pad; row += gridDim.x * blockDim.x) {
        const int slice = row >> 5, lane = row & 31;
        const int64_t st = A.slice_ptr[slice];
        const int w = (int)((A.slice_ptr[slice + 1] - st) >> 5);
        const double s = row_dot<double, double>(A, st, w, lane, p);
        if (row < A.nrows) { q[row] = s; acc = fma(p[row], s, acc); }
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void reduce_kernel(const double* __restrict__ partial, int nvals, double* __restrict__ scal, int op) {
    // one block: sums partial[0..nvals) (and partial[nvals..2 nvals) for the two-dot form)
    __shared__ double sh[2][RED_THREADS];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nvals; i += blockDim.x) {
        a += partial[i];
        if (op == SC_BETA_FCG) b += partial[nvals + i];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double v = sh[0][0], v2 = sh[1][0];
    switch (op) {
        case SC_ALPHA:   scal[S_PQ] = v; scal[S_ALPHA] = v != 0.0 ? scal[S_RZ] / v : 0.0; break;
        case SC_BETA_CG: scal[S_RZ_NEW] = v; scal[S_BETA] = v / scal[S_RZ]; scal[S_RZ] = v; break;
        case SC_BETA_FCG: scal[S_RZ_NEW] = v; scal[S_ZROLD] = v2; scal[S_BETA] = (v - v2) / scal[S_RZ]; scal[S_RZ] = v; break;
        case SC_RZ:      scal[S_RZ] = v; break;
        default: scal[S_TMP] = v; break;
    }
}

__global__ void __launch_bounds__(RED_THREADS) cg_update_kernel(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                                               double* __restrict__ r_old, const double* __restrict__ p,
                                                               const double* __restrict__ q, const double* __restrict__ scal,
                                                               double* __restrict__ partial) {
    const double alpha = scal[S_ALPHA];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = r[i];
        if (r_old) r_old[i] = ri;
        const double rn = fma(-alpha, q[i], ri);
        r[i] = rn;
        acc = fma(rn, rn, acc);
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(RED_THREADS) dot2_kernel(int64_t n, const double* __restrict__ r, const double* __restrict__ z,
                                                          const double* __restrict__ r_old, double* __restrict__ partial) {
    double a = 0.0, b = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double zi = z[i];
        a = fma(r[i], zi, a);
        if (r_old) b = fma(r_old[i], zi, b);
    }
    const double ta = block_sum(a);
    if (threadIdx.x == 0) partial[blockIdx.x] = ta;
    if (r_old) {
        const double tb = block_sum(b);
        if (threadIdx.x == 0) partial[gridDim.x + blockIdx.x] = tb;
    }
}

__global__ void p_update_kernel(int64_t n, double* __restrict__ p, const double* __restrict__ z,
                                const double* __restrict__ scal) {
    const double beta = scal[S_BETA];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
}

__global__ void pcg_check_kernel(cudaGraphConditionalHandle hw, double* __restrict__ scal, int* __restrict__ iter,
                                 double tol, int maxit) {
    const int k = ++iter[0];
    const double r0 = scal[S_R0];
    const double rel = r0 > 0.0 ? sqrt(scal[S_TMP]) / r0 : 0.0;
    scal[S_REL] = rel;
    const bool go = (rel > tol) && (k < maxit);   // a NaN residual stops the loop
    cudaGraphSetConditional(hw, go ? 1u : 0u);
}

__global__ void pcg_start_kernel(double* __restrict__ scal, int* __restrict__ iter) {
    scal[S_R0] = sqrt(scal[S_TMP]);
    scal[S_REL] = 1.0;
    iter[0] = 0;
}

template <class T>
__global__ void to_double_kernel(const T* __restrict__ in, double* __restrict__ out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}

__global__ void axpy1_kernel(int64_t n, double* __restrict__ x, const double* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += y[i];
}

}  // namespace

template <class V, class T>
void launch_sell(int mode, const Sell<V>& A, const T* x, const T* f, const T* dinv, T* y, cudaStream_t s) {
    if (A.nslices == 0) return;
    const int threads = 256;
    const int blocks = (A.nslices * 32 + threads - 1) / threads;
    auto v = view(A);
    switch (mode) {
        case SELL_AX: sell_kernel<V, T, SELL_AX><<<blocks, threads, 0, s>>>(v, x, f, dinv, y); break;
        case SELL_RESID: sell_kernel<V, T, SELL_RESID><<<blocks, threads, 0, s>>>(v, x, f, dinv, y); break;
        case SELL_L1: sell_kernel<V, T, SELL_L1><<<blocks, threads, 0, s>>>(v, x, f, dinv, y); break;
        default: sell_kernel<V, T, SELL_ADD><<<blocks, threads, 0, s>>>(v, x, f, dinv, y); break;
    }
    AMGH_LAUNCHED();
}

template <class T>
void launch_coarse_apply(const T* inv, int n, const T* x, T* y, cudaStream_t s) {
    coarse_apply_kernel<T><<<(n + 7) / 8, 256, 0, s>>>(inv, n, x, y);
    AMGH_LAUNCHED();
}

void launch_spmv_dot(const Sell<double>& A, const double* p, double* q, double* partial, cudaStream_t s) {
    spmv_dot_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(view(A), p, q, partial);
    AMGH_LAUNCHED();
}

void launch_reduce(const double* partial, int nvals, double* scal, int op, cudaStream_t s) {
    reduce_kernel<<<1, RED_THREADS, 0, s>>>(partial, nvals, scal, op);
    AMGH_LAUNCHED();
}

void launch_cg_update(int64_t n, double* x, double* r, double* r_old, const double* p, const double* q,
                      const double* scal, double* partial, cudaStream_t s) {
    cg_update_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, x, r, r_old, p, q, scal, partial);
    AMGH_LAUNCHED();
}

void launch_dot2(int64_t n, const double* r, const double* z, const double* r_old, double* partial, cudaStream_t s) {
    dot2_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, r, z, r_old, partial);
    AMGH_LAUNCHED();
}

void launch_dot(int64_t n, const double* a, const double* b, double* partial, cudaStream_t s) {
    dot2_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, a, b, nullptr, partial);
    AMGH_LAUNCHED();
}

void launch_p_update(int64_t n, double* p, const double* z, const double* scal, cudaStream_t s) {
    p_update_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, p, z, scal);
    AMGH_LAUNCHED();
}

void launch_axpy1(int64_t n, double* x, const double* y, cudaStream_t s) {
    axpy1_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, x, y);
    AMGH_LAUNCHED();
}

void launch_pcg_check(cudaGraphConditionalHandle hw, double* scal, int* iter, double tol, int maxit, cudaStream_t s) {
    pcg_check_kernel<<<1, 1, 0, s>>>(hw, scal, iter, tol, maxit);
    AMGH_LAUNCHED();
}

void launch_pcg_start(double* scal, int* iter, cudaStream_t s) {
    pcg_start_kernel<<<1, 1, 0, s>>>(scal, iter);
    AMGH_LAUNCHED();
}

template <class T>
void launch_to_double(const T* in, double* out, int64_t n, cudaStream_t s) {
    if (n == 0) return;
    to_double_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
    AMGH_LAUNCHED();
}
template void launch_to_double<float>(const float*, double*, int64_t, cudaStream_t);
template void launch_to_double<double>(const double*, double*, int64_t, cudaStream_t);

template void launch_sell<double, double>(int, const Sell<double>&, const double*, const double*, const double*, double*, cudaStream_t);
template void launch_coarse_apply<double>(const double*, int, const double*, double*, cudaStream_t);
template void launch_coarse_apply<float>(const float*, int, const float*, float*, cudaStream_t);

}  // namespace amgh
