// Multi-right-hand-side kernels: K systems that share the matrix, vectors row-major with a
// padded width KP (a multiple of 32).  A level stores its values and vectors in FP64, or in FP32
// with FP32 accumulation; products between levels of different types accumulate in FP64.  A warp owns a matrix row; its lanes own KP/32 consecutive
// columns each, so every gathered vector row is one coalesced read and each nonzero is read once
// for all K right-hand sides.
#include <algorithm>
#include <type_traits>

#include "multi.cuh"
#include "star_invert.cuh"

namespace amgh {

namespace {

// row entries are read 32 at a time by the lanes and broadcast by shuffles, so that the gathers
// of several entries are in flight together
// accumulation type: FP64 when either vector type is FP64
template <class TX, class TY>
using MAcc = typename std::conditional<(sizeof(TX) == 8 || sizeof(TY) == 8), double, float>::type;

template <int KPL, class V, class TX, class TA>
__device__ __forceinline__ void row_times_block(int rb, int re, const int32_t* __restrict__ idx,
                                                const V* __restrict__ val, int KP, int cb, int lane,
                                                const TX* X, TA (&acc)[KPL]) {
    for (int e0 = rb; e0 < re; e0 += 32) {
        const int e = e0 + lane;
        const int myc = e < re ? idx[e] : 0;
        const TA myv = e < re ? (TA)val[e] : TA(0);
        const int cnt = min(32, re - e0);
#pragma unroll 8
        for (int q = 0; q < cnt; ++q) {
            const int c = __shfl_sync(0xffffffffu, myc, q);
            const TA v = __shfl_sync(0xffffffffu, myv, q);
            const TX* xr = X + (int64_t)c * KP + cb + lane * KPL;
#pragma unroll
            for (int j = 0; j < KPL; ++j) acc[j] = fma(v, (TA)xr[j], acc[j]);
        }
    }
}

template <int KPL, int MODE, class V, class TX, class TY>
__global__ void __launch_bounds__(256) spmm_kernel(int n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                                   const V* __restrict__ val, int KP, const TX* __restrict__ X,
                                                   const TY* __restrict__ F, const TY* __restrict__ dinv,
                                                   TY* __restrict__ Y) {
    using TA = MAcc<TX, TY>;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= n) return;
    const int cb = blockIdx.y * 32 * KPL;
    TA acc[KPL];
#pragma unroll
    for (int j = 0; j < KPL; ++j) acc[j] = TA(0);
    row_times_block<KPL, V, TX, TA>(ptr[row], ptr[row + 1], idx, val, KP, cb, lane, X, acc);
    const int64_t o = (int64_t)row * KP + cb + lane * KPL;
#pragma unroll
    for (int j = 0; j < KPL; ++j) {
        if (MODE == MM_AX) Y[o + j] = (TY)acc[j];
        else if (MODE == MM_RESID) Y[o + j] = (TY)((TA)F[o + j] - acc[j]);
        else if (MODE == MM_L1) Y[o + j] = (TY)((TA)X[o + j] + (TA)dinv[row] * ((TA)F[o + j] - acc[j]));
        else Y[o + j] = (TY)((TA)Y[o + j] + acc[j]);
    }
}

// columns per lane: the largest of 8, 4, 2, 1 that divides KP / 32
inline int lane_width(int KP) {
    const int m = KP / 32;
    for (int k : {8, 4, 2}) if (m % k == 0) return k;
    return 1;
}

template <int MODE, class V, class TX, class TY>
void spmm_mode(int nrows, const int32_t* ptr, const int32_t* idx, const V* val, int KP, const TX* X, const TY* F,
               const TY* dinv, TY* Y, cudaStream_t s) {
    const int kpl = lane_width(KP);
    dim3 grid((unsigned)(((int64_t)nrows * 32 + 255) / 256), (unsigned)(KP / (32 * kpl)));
    switch (kpl) {
        case 1: spmm_kernel<1, MODE, V, TX, TY><<<grid, 256, 0, s>>>(nrows, ptr, idx, val, KP, X, F, dinv, Y); break;
        case 2: spmm_kernel<2, MODE, V, TX, TY><<<grid, 256, 0, s>>>(nrows, ptr, idx, val, KP, X, F, dinv, Y); break;
        case 4: spmm_kernel<4, MODE, V, TX, TY><<<grid, 256, 0, s>>>(nrows, ptr, idx, val, KP, X, F, dinv, Y); break;
        default: spmm_kernel<8, MODE, V, TX, TY><<<grid, 256, 0, s>>>(nrows, ptr, idx, val, KP, X, F, dinv, Y); break;
    }
}

// One colour of the multi-RHS Schwarz sweep: a CTA per (star, chunk of 32 KPL columns), a warp
// per row of the star.  Each warp forms F - A X for its row on the chunk into shared memory; after
// a barrier each warp adds its row of A_BB^{-1} applied to the star's residuals.
template <int KPL, class T>
__global__ void __launch_bounds__(256) schwarz_multi_kernel(const int32_t* __restrict__ Aptr, const int32_t* __restrict__ Aidx,
                                                            const T* __restrict__ Aval, const int32_t* __restrict__ stars,
                                                            const int32_t* __restrict__ sptr, const int32_t* __restrict__ sidx,
                                                            const int64_t* __restrict__ ioff, const T* __restrict__ inv,
                                                            int KP, const T* __restrict__ F, T* __restrict__ X) {
    extern __shared__ __align__(16) unsigned char mr_dyn[];
    T* R = reinterpret_cast<T*>(mr_dyn);   // b x (32 KPL)
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = stars[blockIdx.x];
    const int cb = blockIdx.y * 32 * KPL;
    const int b0 = sptr[j], b = sptr[j + 1] - b0;
    for (int q = wl; q < b; q += MR_WARPS) {
        const int row = sidx[b0 + q];
        T acc[KPL];
#pragma unroll
        for (int t = 0; t < KPL; ++t) acc[t] = T(0);
        row_times_block<KPL, T, T, T>(Aptr[row], Aptr[row + 1], Aidx, Aval, KP, cb, lane, X, acc);
        const T* fr = F + (int64_t)row * KP + cb + lane * KPL;
#pragma unroll
        for (int t = 0; t < KPL; ++t) R[q * 32 * KPL + lane * KPL + t] = fr[t] - acc[t];
    }
    __syncthreads();
    const T* iv = inv + ioff[j];
    for (int q = wl; q < b; q += MR_WARPS) {
        const int row = sidx[b0 + q];
        T d[KPL];
#pragma unroll
        for (int t = 0; t < KPL; ++t) d[t] = T(0);
        for (int k = 0; k < b; ++k) {
            const T a = iv[q * b + k];
#pragma unroll
            for (int t = 0; t < KPL; ++t) d[t] = fma(a, R[k * 32 * KPL + lane * KPL + t], d[t]);
        }
        T* xr = X + (int64_t)row * KP + cb + lane * KPL;
#pragma unroll
        for (int t = 0; t < KPL; ++t) xr[t] += d[t];
    }
}

// Split-K form of one colour step for levels with long rows: a CTA per (row of the colour, column
// chunk); its 8 warps take every 8th group of 32 entries of the row, and the partial sums meet in
// shared memory in a fixed order.  R_c[t] = F[row_t] - A[row_t, :] X on the chunk.
template <int KPL, class T>
__global__ void __launch_bounds__(256) multi_resid_splitk_kernel(const int32_t* __restrict__ Aptr,
                                                                 const int32_t* __restrict__ Aidx,
                                                                 const T* __restrict__ Aval,
                                                                 const int32_t* __restrict__ rows, int KP,
                                                                 const T* __restrict__ F,
                                                                 const T* __restrict__ X, T* __restrict__ Rc) {
    __shared__ T part[MR_WARPS][32 * KPL];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x, row = rows[t];
    const int cb = blockIdx.y * 32 * KPL;
    T acc[KPL];
#pragma unroll
    for (int j = 0; j < KPL; ++j) acc[j] = T(0);
    const int rb = Aptr[row], re = Aptr[row + 1];
    for (int e0 = rb + 32 * wl; e0 < re; e0 += 32 * MR_WARPS) {
        const int e = e0 + lane;
        const int myc = e < re ? Aidx[e] : 0;
        const T myv = e < re ? Aval[e] : T(0);
        const int cnt = min(32, re - e0);
#pragma unroll 8
        for (int q = 0; q < cnt; ++q) {
            const int c = __shfl_sync(0xffffffffu, myc, q);
            const T v = __shfl_sync(0xffffffffu, myv, q);
            const T* xr = X + (int64_t)c * KP + cb + lane * KPL;
#pragma unroll
            for (int j = 0; j < KPL; ++j) acc[j] = fma(v, xr[j], acc[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < KPL; ++j) part[wl][lane * KPL + j] = acc[j];
    __syncthreads();
    for (int i = threadIdx.x; i < 32 * KPL; i += 32 * MR_WARPS) {
        T s = T(0);
#pragma unroll
        for (int w = 0; w < MR_WARPS; ++w) s += part[w][i];
        Rc[(int64_t)t * KP + cb + i] = F[(int64_t)row * KP + cb + i] - s;
    }
}

// x_B += A_BB^{-1} r_B, a warp per (row of the colour, column chunk); the star's residual rows are
// consecutive in R_c starting at the star's base
template <int KPL, class T>
__global__ void __launch_bounds__(256) multi_apply_kernel(int nrows_c, const int32_t* __restrict__ rows,
                                                          const int32_t* __restrict__ rstar,
                                                          const int32_t* __restrict__ rq,
                                                          const int32_t* __restrict__ rbase,
                                                          const int32_t* __restrict__ sptr,
                                                          const int64_t* __restrict__ ioff,
                                                          const T* __restrict__ inv, int KP,
                                                          const T* __restrict__ Rc, T* __restrict__ X) {
    const int t = blockIdx.x * MR_WARPS + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (t >= nrows_c) return;
    const int cb = blockIdx.y * 32 * KPL;
    const int j = rstar[t], q = rq[t], base = rbase[t];
    const int b = sptr[j + 1] - sptr[j];
    const T* iv = inv + ioff[j] + (int64_t)q * b;
    T d[KPL];
#pragma unroll
    for (int u = 0; u < KPL; ++u) d[u] = T(0);
    for (int k = 0; k < b; ++k) {
        const T a = iv[k];
        const T* rr = Rc + (int64_t)(base + k) * KP + cb + lane * KPL;
#pragma unroll
        for (int u = 0; u < KPL; ++u) d[u] = fma(a, rr[u], d[u]);
    }
    T* xr = X + (int64_t)rows[t] * KP + cb + lane * KPL;
#pragma unroll
    for (int u = 0; u < KPL; ++u) xr[u] += d[u];
}

__global__ void star_inverse_rm_kernel(const int32_t* __restrict__ Aptr, const int32_t* __restrict__ Aidx,
                                       const double* __restrict__ Aval, int nstars, const int32_t* __restrict__ star_ptr,
                                       const int32_t* __restrict__ star_idx, const int64_t* __restrict__ ioff,
                                       double* __restrict__ inv, int* err_flag) {
    __shared__ double sm[2][2][32 * 33];
    __shared__ double fac[2][32];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * 2 + wl;
    if (j >= nstars) return;
    const int b0 = star_ptr[j], b = star_ptr[j + 1] - b0;
    if (b == 0) return;
    const bool ok = star_invert(Aptr, Aidx, Aval, star_idx, b0, b, sm[wl][0], sm[wl][1], fac[wl]);
    if (!ok && lane == 0) atomicExch(err_flag, 1);
    if (lane < b)
        for (int k = 0; k < b; ++k) inv[ioff[j] + lane * b + k] = sm[wl][1][lane * 33 + k];
}

template <class TX, class TY>
__global__ void dense_apply_multi_kernel(const double* __restrict__ Ainv, int n, int KP, const TX* __restrict__ X,
                                         TY* __restrict__ Y) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * KP) return;
    const int i = (int)(t / KP), c = (int)(t % KP);
    double s = 0.0;
    for (int k = 0; k < n; ++k) s = fma(Ainv[(int64_t)i * n + k], (double)X[(int64_t)k * KP + c], s);
    Y[t] = (TY)s;
}

__global__ void widen_kernel(const float* __restrict__ in, int64_t n, double* __restrict__ out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = (double)in[t];
}

__global__ void to_rowmajor_kernel(const double* __restrict__ in, int64_t n, int k, int KP, double* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * KP) return;
    const int64_t i = t / KP;
    const int c = (int)(t % KP);
    out[t] = c < k ? in[(int64_t)c * n + i] : 0.0;
}

__global__ void to_colmajor_kernel(const double* __restrict__ in, int64_t n, int k, int KP, double* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * (int64_t)k) return;
    const int c = (int)(t / n);
    const int64_t i = t % n;
    out[t] = in[i * KP + c];
}

constexpr int CD_BLOCKS = 304;

// per-column partial sums over a fixed set of row ranges (deterministic order)
__global__ void coldot_partial_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n, int KP,
                                      double* __restrict__ partial) {
    extern __shared__ double sh[];
    const int tid = threadIdx.x;
    const int64_t rows_per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * rows_per, r1 = std::min<int64_t>(n, r0 + rows_per);
    for (int c0 = 0; c0 < KP; c0 += blockDim.x) {
        const int c = c0 + tid;
        double s = 0.0;
        if (c < KP)
            for (int64_t r = r0; r < r1; ++r) s = fma(a[r * KP + c], b[r * KP + c], s);
        if (c < KP) partial[(int64_t)blockIdx.x * KP + c] = s;
    }
    (void)sh;
}

__global__ void coldot_final_kernel(const double* __restrict__ partial, int nb, int KP, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= KP) return;
    double s = 0.0;
    for (int q = 0; q < nb; ++q) s += partial[(int64_t)q * KP + c];
    out[c] = s;
}

__global__ void mcg_update_kernel(int64_t total, int KP, double* __restrict__ X, double* __restrict__ R,
                                  double* __restrict__ Rold, const double* __restrict__ P, const double* __restrict__ Q,
                                  const double* __restrict__ alpha) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const double a = alpha[t % KP];
        X[t] = fma(a, P[t], X[t]);
        const double r = R[t];
        if (Rold) Rold[t] = r;
        R[t] = fma(-a, Q[t], r);
    }
}

__global__ void mp_update_kernel(int64_t total, int KP, double* __restrict__ P, const double* __restrict__ Z,
                                 const double* __restrict__ beta) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        P[t] = fma(beta[t % KP], P[t], Z[t]);
}


}  // namespace

template <class V, class TX, class TY>
void launch_spmm_t(int mode, int nrows, const int32_t* ptr, const int32_t* idx, const V* val, int KP, const TX* X,
                   const TY* F, const TY* dinv, TY* Y, cudaStream_t s) {
    if (nrows == 0) return;
    switch (mode) {
        case MM_AX: spmm_mode<MM_AX>(nrows, ptr, idx, val, KP, X, F, dinv, Y, s); break;
        case MM_RESID: spmm_mode<MM_RESID>(nrows, ptr, idx, val, KP, X, F, dinv, Y, s); break;
        case MM_L1: spmm_mode<MM_L1>(nrows, ptr, idx, val, KP, X, F, dinv, Y, s); break;
        default: spmm_mode<MM_ADD>(nrows, ptr, idx, val, KP, X, F, dinv, Y, s); break;
    }
    AMGH_LAUNCHED();
}

void launch_spmm(int mode, const DevCSR& M, int KP, const double* X, const double* F, const double* dinv, double* Y,
                 cudaStream_t s) {
    launch_spmm_t<double, double, double>(mode, M.nrows, M.ptr.p, M.idx.p, M.val.p, KP, X, F, dinv, Y, s);
}

template <class T>
void launch_schwarz_multi_t(const MultiLevel& L, const T* Aval, const T* inv, T* Rc, int colour, int KP, const T* F,
                            T* X, cudaStream_t s) {
    const int sb = L.colour_star_begin[colour], se = L.colour_star_begin[colour + 1];
    const int nst = se - sb;
    if (nst <= 0) return;
    const int kpl = lane_width(KP);
    if (L.splitk) {
        const int r0 = L.colour_row_begin[colour], nr = L.colour_row_begin[colour + 1] - r0;
        if (nr <= 0) return;
        // narrower column chunks when the colour has few rows, so that a step fills the GPU
        int kpl_s = kpl;
        while (kpl_s > 1 && (int64_t)nr * (KP / (32 * kpl_s)) < 4 * 152) kpl_s >>= 1;
        const int kpl = kpl_s;
        const unsigned chunks = (unsigned)(KP / (32 * kpl));
        dim3 g1((unsigned)nr, chunks), g2((unsigned)((nr + MR_WARPS - 1) / MR_WARPS), chunks);
#define AMGH_SK(K)                                                                                                 \
    multi_resid_splitk_kernel<K, T><<<g1, 32 * MR_WARPS, 0, s>>>(L.A->ptr.p, L.A->idx.p, Aval, L.crow.p + r0, KP, F, X, \
                                                                Rc);                                                    \
    multi_apply_kernel<K, T><<<g2, 32 * MR_WARPS, 0, s>>>(nr, L.crow.p + r0, L.cstar.p + r0, L.cq.p + r0,               \
                                                         L.cbase.p + r0, L.star_ptr.p, L.inv_off.p, inv, KP, Rc, X);
        switch (kpl) {
            case 1: AMGH_SK(1) break;
            case 2: AMGH_SK(2) break;
            case 4: AMGH_SK(4) break;
            default: AMGH_SK(8) break;
        }
#undef AMGH_SK
        AMGH_LAUNCHED();
        AMGH_LAUNCHED();
        return;
    }
    const size_t shm = (size_t)L.bmax * 32 * kpl * sizeof(T);   // <= 32 x 256 doubles = 64 KB
    dim3 grid((unsigned)nst, (unsigned)(KP / (32 * kpl)));
    const int32_t* stars = L.star_list.p + sb;
#define AMGH_SM(K)                                                                                                        \
    AMGH_CUDA(cudaFuncSetAttribute(schwarz_multi_kernel<K, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm)); \
    schwarz_multi_kernel<K, T><<<grid, 256, shm, s>>>(L.A->ptr.p, L.A->idx.p, Aval, stars, L.star_ptr.p, L.star_idx.p,   \
                                                      L.inv_off.p, inv, KP, F, X);
    switch (kpl) {
        case 1: AMGH_SM(1) break;
        case 2: AMGH_SM(2) break;
        case 4: AMGH_SM(4) break;
        default: AMGH_SM(8) break;
    }
#undef AMGH_SM
    AMGH_LAUNCHED();
}

void launch_star_inverse_rowmajor(const DevCSR& A, int nstars, const int32_t* star_ptr, const int32_t* star_idx,
                                  const int64_t* inv_off, double* inv, int* err_flag, cudaStream_t s) {
    if (nstars == 0) return;
    star_inverse_rm_kernel<<<(nstars + 1) / 2, 64, 0, s>>>(A.ptr.p, A.idx.p, A.val.p, nstars, star_ptr, star_idx, inv_off,
                                                           inv, err_flag);
    AMGH_LAUNCHED();
}

template <class TX, class TY>
void launch_dense_apply_multi_t(const double* Ainv, int n, int KP, const TX* X, TY* Y, cudaStream_t s) {
    const int64_t total = (int64_t)n * KP;
    if (total == 0) return;
    dense_apply_multi_kernel<TX, TY><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Ainv, n, KP, X, Y);
    AMGH_LAUNCHED();
}

void launch_widen(const float* in, int64_t n, double* out, cudaStream_t s) {
    if (n == 0) return;
    widen_kernel<<<608, 256, 0, s>>>(in, n, out);
    AMGH_LAUNCHED();
}

#define INST_MSPMM(V, TX, TY)                                                                                     \
    template void launch_spmm_t<V, TX, TY>(int, int, const int32_t*, const int32_t*, const V*, int, const TX*,   \
                                           const TY*, const TY*, TY*, cudaStream_t);
INST_MSPMM(double, double, double)
INST_MSPMM(float, float, float)
INST_MSPMM(double, double, float)
INST_MSPMM(float, float, double)
INST_MSPMM(double, float, double)
INST_MSPMM(float, double, float)
template void launch_schwarz_multi_t<double>(const MultiLevel&, const double*, const double*, double*, int, int,
                                             const double*, double*, cudaStream_t);
template void launch_schwarz_multi_t<float>(const MultiLevel&, const float*, const float*, float*, int, int,
                                            const float*, float*, cudaStream_t);
template void launch_dense_apply_multi_t<double, double>(const double*, int, int, const double*, double*, cudaStream_t);
template void launch_dense_apply_multi_t<float, float>(const double*, int, int, const float*, float*, cudaStream_t);

void launch_to_rowmajor(const double* in, int64_t n, int k, int KP, double* out, cudaStream_t s) {
    const int64_t total = n * KP;
    if (total == 0) return;
    to_rowmajor_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(in, n, k, KP, out);
    AMGH_LAUNCHED();
}

void launch_to_colmajor(const double* in, int64_t n, int k, int KP, double* out, cudaStream_t s) {
    const int64_t total = n * k;
    if (total == 0) return;
    to_colmajor_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(in, n, k, KP, out);
    AMGH_LAUNCHED();
}

void launch_coldot(const double* a, const double* b, int64_t n, int KP, double* partial, double* out, cudaStream_t s) {
    coldot_partial_kernel<<<CD_BLOCKS, 256, 0, s>>>(a, b, n, KP, partial);
    AMGH_LAUNCHED();
    coldot_final_kernel<<<(KP + 255) / 256, 256, 0, s>>>(partial, CD_BLOCKS, KP, out);
    AMGH_LAUNCHED();
}

void launch_mcg_update(int64_t n, int KP, double* X, double* R, double* Rold, const double* P, const double* Q,
                       const double* alpha, cudaStream_t s) {
    mcg_update_kernel<<<608, 256, 0, s>>>(n * KP, KP, X, R, Rold, P, Q, alpha);
    AMGH_LAUNCHED();
}

void launch_mp_update(int64_t n, int KP, double* P, const double* Z, const double* beta, cudaStream_t s) {
    mp_update_kernel<<<608, 256, 0, s>>>(n * KP, KP, P, Z, beta);
    AMGH_LAUNCHED();
}


}  // namespace amgh
