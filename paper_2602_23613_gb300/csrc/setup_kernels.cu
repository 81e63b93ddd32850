// Setup numerics on the device (FP64): local harmonic-extension solves (Eq. sparseP), Galerkin
// product (Eq. tl), star-block and coarsest inverses, l1 row norms, SELL layouts.
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.h"

namespace amgh {

namespace {

__device__ __forceinline__ int bsearch_i32(const int32_t* __restrict__ a, int lo, int hi, int key) {
    // position of key in a[lo, hi) (ascending) or -1
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = a[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid;
    }
    return -1;
}

template <class V> __device__ __forceinline__ V from_double(double x);
template <> __device__ __forceinline__ double from_double<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_double<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double x) {
    return __float2bfloat16_rn((float)x);
}

// ---------------------------------------------------------------------------------------------
// One CTA per coarse edge: gather the lower triangle of A_pp (packed, row i at i(i+1)/2) and the
// right-hand side -(A_{p,d1} s1 + A_{p,d2} s2) into shared memory; factor A_pp = L D L^T in place
// by right-looking elimination with one barrier per pivot (step k reads column k and updates the
// trailing lower triangle, so no entry is read and written in the same step); then one warp runs
// the two triangular solves and the diagonal scaling; scatter into P and P^T.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int tri(int i) { return i * (i + 1) / 2; }

__global__ void patch_solve_kernel(const int32_t* __restrict__ Aptr, const int32_t* __restrict__ Aidx,
                                   const double* __restrict__ Aval, int c0, int nc,
                                   const int32_t* __restrict__ edges4, const int32_t* __restrict__ patch_ptr,
                                   const int32_t* __restrict__ patch_idx, const int64_t* __restrict__ pos_P,
                                   const int64_t* __restrict__ pos_PT, double* __restrict__ Pval,
                                   double* __restrict__ PTval, int max_patch, int* err_flag) {
    extern __shared__ double smem[];
    const int c = c0 + blockIdx.x;
    if (c >= nc) return;
    const int p0 = patch_ptr[c];
    const int m = patch_ptr[c + 1] - p0;
    if (m == 0) return;
    double* L = smem;                                // packed lower triangle, tri(max_patch) entries
    double* y = smem + tri(max_patch);
    double* dinv = y + max_patch;
    int* pidx = reinterpret_cast<int*>(dinv + max_patch);
    __shared__ int bad;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    if (tid == 0) bad = 0;
    for (int a = tid; a < m; a += nt) pidx[a] = patch_idx[p0 + a];
    for (int e = tid; e < tri(m); e += nt) L[e] = 0.0;
    __syncthreads();
    const int d1 = edges4[4 * c], s1 = edges4[4 * c + 1], d2 = edges4[4 * c + 2], s2 = edges4[4 * c + 3];
    for (int a = tid; a < m; a += nt) {
        const int g = pidx[a];
        const int rb = Aptr[g], re = Aptr[g + 1];
        for (int q = rb; q < re; ++q) {
            const int b = bsearch_i32(pidx, 0, a + 1, Aidx[q]);
            if (b >= 0) L[tri(a) + b] = Aval[q];
        }
        const int q1 = bsearch_i32(Aidx, rb, re, d1);
        const int q2 = bsearch_i32(Aidx, rb, re, d2);
        double rhs = 0.0;
        if (q1 >= 0) rhs -= Aval[q1] * (double)s1;
        if (q2 >= 0) rhs -= Aval[q2] * (double)s2;
        y[a] = rhs;
    }
    // L D L^T: after step k, L[k][k] = d_k and L[i][k] = l_ik d_k for i > k
    for (int k = 0; k < m; ++k) {
        __syncthreads();
        const double piv = L[tri(k) + k];
        if (!(piv > 0.0)) {
            if (tid == 0) bad = 1;
            continue;
        }
        const double inv = 1.0 / piv;
        if (tid == 0) dinv[k] = inv;
        for (int i = k + 1 + warp; i < m; i += nw) {
            const double lik = L[tri(i) + k] * inv;
            double* Li = L + tri(i);
            for (int j = k + 1 + lane; j <= i; j += 32) Li[j] -= lik * L[tri(j) + k];
        }
    }
    __syncthreads();
    if (bad) {
        if (tid == 0) atomicExch(err_flag, 1);
        return;
    }
    if (warp == 0) {
        // L' z = y with L'[i][k] = L[i][k] d_k^-1, then w = D^-1 z, then L'^T x = w
        for (int k = 0; k < m; ++k) {
            __syncwarp();
            const double zk = y[k] * dinv[k];
            for (int i = k + 1 + lane; i < m; i += 32) y[i] -= L[tri(i) + k] * zk;
        }
        __syncwarp();
        for (int k = lane; k < m; k += 32) y[k] *= dinv[k];
        for (int k = m - 1; k >= 0; --k) {
            __syncwarp();
            const double xk = y[k];
            for (int i = lane; i < k; i += 32) y[i] -= L[tri(k) + i] * dinv[i] * xk;
        }
        __syncwarp();
        for (int a = lane; a < m; a += 32) {
            Pval[pos_P[p0 + a]] = y[a];
            PTval[pos_PT[p0 + a]] = y[a];
        }
    }
}

// Small patches (at most WARP_PATCH DoFs): a warp per coarse edge, four per CTA, the same
// L D L^T factorisation and solves with warp-level synchronisation only; each lane owns the rows
// i = lane, lane + 32 of the trailing update.
constexpr int WARP_PATCH = 48;

constexpr int PATCH_WARPS = 4;   // 4 x 10.4 KB of static shared memory per CTA

__global__ void __launch_bounds__(32 * PATCH_WARPS) patch_solve_warp_kernel(
    const int32_t* __restrict__ Aptr, const int32_t* __restrict__ Aidx, const double* __restrict__ Aval, int c0,
    int nc, const int32_t* __restrict__ edges4, const int32_t* __restrict__ patch_ptr,
    const int32_t* __restrict__ patch_idx, const int64_t* __restrict__ pos_P, const int64_t* __restrict__ pos_PT,
    double* __restrict__ Pval, double* __restrict__ PTval, int* err_flag) {
    constexpr int TRI = WARP_PATCH * (WARP_PATCH + 1) / 2;
    __shared__ double Ls[PATCH_WARPS][TRI];
    __shared__ double ys[PATCH_WARPS][WARP_PATCH], dis[PATCH_WARPS][WARP_PATCH];
    __shared__ int ps[PATCH_WARPS][WARP_PATCH];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = c0 + blockIdx.x * PATCH_WARPS + w;
    if (c >= nc) return;
    const int p0 = patch_ptr[c];
    const int m = patch_ptr[c + 1] - p0;
    if (m == 0) return;
    double* L = Ls[w];
    double* y = ys[w];
    double* dinv = dis[w];
    int* pidx = ps[w];
    for (int a = lane; a < m; a += 32) pidx[a] = patch_idx[p0 + a];
    for (int e = lane; e < tri(m); e += 32) L[e] = 0.0;
    __syncwarp();
    const int d1 = edges4[4 * c], s1 = edges4[4 * c + 1], d2 = edges4[4 * c + 2], s2 = edges4[4 * c + 3];
    for (int a = lane; a < m; a += 32) {
        const int g = pidx[a];
        const int rb = Aptr[g], re = Aptr[g + 1];
        for (int q = rb; q < re; ++q) {
            const int b = bsearch_i32(pidx, 0, a + 1, Aidx[q]);
            if (b >= 0) L[tri(a) + b] = Aval[q];
        }
        const int q1 = bsearch_i32(Aidx, rb, re, d1);
        const int q2 = bsearch_i32(Aidx, rb, re, d2);
        double rhs = 0.0;
        if (q1 >= 0) rhs -= Aval[q1] * (double)s1;
        if (q2 >= 0) rhs -= Aval[q2] * (double)s2;
        y[a] = rhs;
    }
    bool bad = false;
    for (int k = 0; k < m; ++k) {
        __syncwarp();
        const double piv = L[tri(k) + k];
        if (!(piv > 0.0)) {
            bad = true;
            break;
        }
        const double inv = 1.0 / piv;
        if (lane == 0) dinv[k] = inv;
        for (int i = k + 1 + lane; i < m; i += 32) {
            const double lik = L[tri(i) + k] * inv;
            double* Li = L + tri(i);
            for (int j = k + 1; j <= i; ++j) Li[j] -= lik * L[tri(j) + k];
        }
    }
    if (bad) {
        if (lane == 0) atomicExch(err_flag, 1);
        return;
    }
    for (int k = 0; k < m; ++k) {
        __syncwarp();
        const double zk = y[k] * dinv[k];
        for (int i = k + 1 + lane; i < m; i += 32) y[i] -= L[tri(i) + k] * zk;
    }
    __syncwarp();
    for (int k = lane; k < m; k += 32) y[k] *= dinv[k];
    for (int k = m - 1; k >= 0; --k) {
        __syncwarp();
        const double xk = y[k];
        for (int i = lane; i < k; i += 32) y[i] -= L[tri(k) + i] * dinv[i] * xk;
    }
    __syncwarp();
    for (int a = lane; a < m; a += 32) {
        Pval[pos_P[p0 + a]] = y[a];
        PTval[pos_PT[p0 + a]] = y[a];
    }
}

// exterior entries of column c of P (and row c of P^T): s1 at DoF1, s2 at DoF2 (R^T of Alg. 3)
__global__ void ext_scatter_kernel(int nc, const int32_t* __restrict__ edges4, const int64_t* __restrict__ ext_P,
                                   const int64_t* __restrict__ ext_PT, double* __restrict__ Pval,
                                   double* __restrict__ PTval) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const double s1 = (double)edges4[4 * c + 1], s2 = (double)edges4[4 * c + 3];
    Pval[ext_P[2 * c]] = s1;
    Pval[ext_P[2 * c + 1]] = s2;
    PTval[ext_PT[2 * c]] = s1;
    PTval[ext_PT[2 * c + 1]] = s2;
}

// ---------------------------------------------------------------------------------------------
// Galerkin product: warp per output row, lanes over the row's pattern entries; every entry
// sums its terms in ascending order (deterministic).
// ---------------------------------------------------------------------------------------------
__global__ void ap_kernel(int n, const int32_t* __restrict__ Aptr, const int32_t* __restrict__ Aidx,
                          const double* __restrict__ Aval, const int32_t* __restrict__ Pptr,
                          const int32_t* __restrict__ Pidx, const double* __restrict__ Pval,
                          const int32_t* __restrict__ Optr, const int32_t* __restrict__ Oidx,
                          double* __restrict__ Oval) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int ob = Optr[warp], oe = Optr[warp + 1];
    const int ab = Aptr[warp], ae = Aptr[warp + 1];
    for (int o = ob + lane; o < oe; o += 32) {
        const int J = Oidx[o];
        double s = 0.0;
        for (int q = ab; q < ae; ++q) {
            const int j = Aidx[q];
            const int t = bsearch_i32(Pidx, Pptr[j], Pptr[j + 1], J);
            if (t >= 0) s += Aval[q] * Pval[t];
        }
        Oval[o] = s;
    }
}

// Row-accumulating numeric product O = A P on O's known pattern: a warp per output row keeps the
// row's columns and running sums in shared memory; for every term A(I, q) in ascending q, the
// lanes take the entries of row q of P (distinct columns, so no two lanes touch one sum) and add
// A(I, q) P(q, J) into the sum of J, found by binary search among the row's columns.  Every sum
// therefore adds its terms in ascending q, as the entry-wise kernel above does.
constexpr int ROWACC_MAX = 8192;

__global__ void ap_rowacc_kernel(int n, const int32_t* __restrict__ Aptr, const int32_t* __restrict__ Aidx,
                                 const double* __restrict__ Aval, const int32_t* __restrict__ Pptr,
                                 const int32_t* __restrict__ Pidx, const double* __restrict__ Pval,
                                 const int32_t* __restrict__ Optr, const int32_t* __restrict__ Oidx,
                                 double* __restrict__ Oval, int stride) {
    extern __shared__ double rsm[];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int row = blockIdx.x * nw + wl;
    if (row >= n) return;   // warp-level synchronisation only
    double* acc = rsm + (size_t)wl * stride;
    int* oc = reinterpret_cast<int*>(rsm + (size_t)nw * stride) + (size_t)wl * stride;
    const int ob = Optr[row], m = Optr[row + 1] - ob;
    for (int i = lane; i < m; i += 32) {
        oc[i] = Oidx[ob + i];
        acc[i] = 0.0;
    }
    const int qb = Aptr[row], qe = Aptr[row + 1];
    for (int q0 = qb; q0 < qe; q0 += 32) {
        const int q = q0 + lane;
        const bool ok = q < qe;
        const int j = ok ? Aidx[q] : 0;
        const double a = ok ? Aval[q] : 0.0;
        const int pb = ok ? Pptr[j] : 0, pe = ok ? Pptr[j + 1] : 0;
        const int cnt = min(32, qe - q0);
        for (int t = 0; t < cnt; ++t) {
            const double at = __shfl_sync(0xffffffffu, a, t);
            const int b = __shfl_sync(0xffffffffu, pb, t), e = __shfl_sync(0xffffffffu, pe, t);
            __syncwarp();
            for (int u = b + lane; u < e; u += 32) {
                const int J = Pidx[u];
                int lo = 0, hi = m;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (oc[mid] < J) lo = mid + 1;
                    else hi = mid;
                }
                acc[lo] = fma(at, Pval[u], acc[lo]);
            }
        }
    }
    __syncwarp();
    for (int i = lane; i < m; i += 32) Oval[ob + i] = acc[i];
}

__global__ void l1inv_kernel_d(int n, const int32_t* __restrict__ ptr, const double* __restrict__ val,
                               double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int q = ptr[i]; q < ptr[i + 1]; ++q) s += fabs(val[q]);
    out[i] = 1.0 / s;
}

template <class T>
__global__ void convert_kernel(const double* __restrict__ in, T* __restrict__ out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = from_double<T>(in[i]);
}
template <>
__global__ void convert_kernel<double>(const double* __restrict__ in, double* __restrict__ out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

template <class V>
__global__ void sell_fill_kernel(int n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                 const double* __restrict__ val, int nslices, const int64_t* __restrict__ sptr,
                                 int32_t* __restrict__ scol, V* __restrict__ sval) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = row >> 5, lane = row & 31;
    if (slice >= nslices) return;
    const int64_t st = sptr[slice];
    const int w = (int)((sptr[slice + 1] - st) >> 5);
    int b = 0, len = 0;
    if (row < n) { b = ptr[row]; len = ptr[row + 1] - b; }
    // padding repeats the row's last column (a valid, nearby column; value 0)
    const int pad_col = len > 0 ? idx[b + len - 1] : 0;
    for (int t = 0; t < w; ++t) {
        const int64_t o = st + 32 * (int64_t)t + lane;
        if (t < len) { scol[o] = idx[b + t]; sval[o] = from_double<V>(val[b + t]); }
        else { scol[o] = pad_col; sval[o] = from_double<V>(0.0); }
    }
}

// Dense inverse of the coarsest matrix, one CTA: gather, Gauss-Jordan (SPD, no pivoting).
__global__ void coarse_inverse_kernel(int n, const int32_t* __restrict__ Aptr, const int32_t* __restrict__ Aidx,
                                      const double* __restrict__ Aval, double* __restrict__ inv,
                                      double* __restrict__ M, int* err_flag) {
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ double piv_s;
    for (int e = tid; e < n * n; e += nt) { M[e] = 0.0; inv[e] = (e / n == e % n) ? 1.0 : 0.0; }
    __syncthreads();
    for (int r = tid; r < n; r += nt)
        for (int q = Aptr[r]; q < Aptr[r + 1]; ++q) M[(int64_t)r * n + Aidx[q]] = Aval[q];
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            double p = M[(int64_t)k * n + k];
            if (!(p > 0.0)) { atomicExch(err_flag, 1); p = 1.0; }
            piv_s = p;
        }
        __syncthreads();
        const double p = piv_s;
        for (int j = tid; j < n; j += nt) { M[(int64_t)k * n + j] /= p; inv[(int64_t)k * n + j] /= p; }
        __syncthreads();
        for (int e = tid; e < n * n; e += nt) {
            const int i = e / n, j = e % n;
            if (i == k) continue;
            const double f = M[(int64_t)i * n + k];
            // column k of M is read by every j of row i: update column k last (j == k handled below)
            if (j != k) {
                M[(int64_t)i * n + j] -= f * M[(int64_t)k * n + j];
            }
            inv[(int64_t)i * n + j] -= f * inv[(int64_t)k * n + j];
        }
        __syncthreads();
        for (int i = tid; i < n; i += nt)
            if (i != k) M[(int64_t)i * n + k] = 0.0;
        __syncthreads();
    }
}

}  // namespace

void launch_ext_scatter(int nc, const int32_t* edges4, const int64_t* ext_P, const int64_t* ext_PT, double* Pval,
                        double* PTval, cudaStream_t s) {
    if (nc == 0) return;
    ext_scatter_kernel<<<(nc + 255) / 256, 256, 0, s>>>(nc, edges4, ext_P, ext_PT, Pval, PTval);
    AMGH_LAUNCHED();
}

void launch_patch_solve(const DevCSR& A, int nc, const int32_t* edges4, const int32_t* patch_ptr,
                        const int32_t* patch_idx, const int64_t* pos_P, const int64_t* pos_PT,
                        double* Pval, double* PTval, int max_patch, int* err_flag, cudaStream_t s) {
    if (nc == 0 || max_patch == 0) return;
    if (max_patch <= WARP_PATCH) {
        const int per = PATCH_WARPS, chunk = 65535 * per;
        for (int c0 = 0; c0 < nc; c0 += chunk) {
            const int cnt = std::min(chunk, nc - c0);
            patch_solve_warp_kernel<<<(cnt + per - 1) / per, 32 * PATCH_WARPS, 0, s>>>(A.ptr.p, A.idx.p, A.val.p, c0, nc, edges4,
                                                                          patch_ptr, patch_idx, pos_P, pos_PT, Pval,
                                                                          PTval, err_flag);
            AMGH_LAUNCHED();
        }
        return;
    }
    const size_t tri_n = (size_t)max_patch * (max_patch + 1) / 2;
    const size_t shm = tri_n * 8 + 2 * (size_t)max_patch * 8 + (size_t)max_patch * 4;
    static_assert(sizeof(int) == 4, "int");
    AMGH_CUDA(cudaFuncSetAttribute(patch_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    const int chunk = 65535;
    for (int c0 = 0; c0 < nc; c0 += chunk) {
        const int cnt = std::min(chunk, nc - c0);
        patch_solve_kernel<<<cnt, 256, shm, s>>>(A.ptr.p, A.idx.p, A.val.p, c0, nc, edges4, patch_ptr, patch_idx,
                                                 pos_P, pos_PT, Pval, PTval, max_patch, err_flag);
        AMGH_LAUNCHED();
    }
}

// Eq. commuting: every interior row p of P (the local extension) moved, on its own pattern, to
// the nearest row satisfying p C = t, C the pattern's rows of G_c on the row's local nodes and t
// row i of 2 G P_n (host-built).  The least-distance change is C y with C^T C y = r, r = t - p C
// taken to the range of C^T C: its mean is removed on every component of the local graph that no
// one-ended row grounds, whose first node is then left out (y = 0 there); C^T C (small integer
// entries) is factored by Cholesky.  One thread per row, its packed matrix and vector in its own
// slice of shared memory; rows come grouped by their number of local nodes, one launch per size
// class M (8 to 128), with as many threads per CTA as keep one or two CTAs per SM.
namespace {

constexpr int COMMUTE_SIZES[5] = {8, 16, 32, 64, 128};

// a thread's slice in doubles, odd so that the threads' 8-byte accesses fall in distinct banks
__host__ __device__ constexpr int commute_slice(int M) { return (M * (M + 1) / 2 + M) | 1; }
// threads per CTA: two CTAs' slices (about 70-140 KB each) per SM where they fit
__host__ __device__ constexpr int commute_threads(int M) {
    return M <= 8 ? 256 : (M <= 16 ? 64 : (M <= 32 ? 24 : (M <= 64 ? 8 : 2)));
}

template <int M>
__global__ void __launch_bounds__(commute_threads(M)) commute_rows_kernel(
    int count, const int32_t* __restrict__ order, const int32_t* __restrict__ rows, const int32_t* __restrict__ Pptr,
    double* __restrict__ Pval, double* __restrict__ PTval, const int32_t* __restrict__ pt_pos,
    const int16_t* __restrict__ ea, const int16_t* __restrict__ eb, const int32_t* __restrict__ node_ptr,
    const double* __restrict__ tt, const int32_t* __restrict__ comp, int* err_flag) {
    extern __shared__ double commute_shm[];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int r = order[k];
    const int i = rows[r];
    const int q0 = Pptr[i], q1 = Pptr[i + 1];
    const int n0 = node_ptr[r], m = node_ptr[r + 1] - n0;
    if (m > M) {   // the host groups rows by size; anything else is an internal error
        atomicExch(err_flag, 1);
        return;
    }
    const int32_t* cp = comp + n0;
    double* L = commute_shm + (size_t)threadIdx.x * commute_slice(M);
    double* y = L + M * (M + 1) / 2;
    for (int u = 0; u < m; ++u) y[u] = tt[n0 + u];
    for (int q = q0; q < q1; ++q) {
        const double p = Pval[q];
        const int a = ea[q], b = eb[q];
        if (a) y[(a > 0 ? a : -a) - 1] -= a > 0 ? p : -p;
        if (b) y[(b > 0 ? b : -b) - 1] -= b > 0 ? p : -p;
    }
    for (int u = 0; u < m; ++u) {
        if (cp[u] != u) continue;   // not the first node of an ungrounded component
        double sum = 0.0;
        int cnt = 0;
        for (int v = u; v < m; ++v)
            if (cp[v] == u) {
                sum += y[v];
                ++cnt;
            }
        const double mean = sum / cnt;
        for (int v = u; v < m; ++v)
            if (cp[v] == u) y[v] -= mean;
    }
    auto at = [](int a, int b) { return a >= b ? a * (a + 1) / 2 + b : b * (b + 1) / 2 + a; };
    for (int t = 0; t < m * (m + 1) / 2; ++t) L[t] = 0.0;
    for (int q = q0; q < q1; ++q) {
        const int a = ea[q], b = eb[q];
        const int la = a ? (a > 0 ? a : -a) - 1 : -1, lb = b ? (b > 0 ? b : -b) - 1 : -1;
        const bool ua = la >= 0 && cp[la] != la, ub = lb >= 0 && cp[lb] != lb;   // in the solve
        if (ua) L[at(la, la)] += 1.0;
        if (ub) L[at(lb, lb)] += 1.0;
        if (ua && ub) L[at(la, lb)] += (a > 0) == (b > 0) ? 1.0 : -1.0;
    }
    for (int u = 0; u < m; ++u)
        if (cp[u] == u) {
            L[at(u, u)] = 1.0;
            y[u] = 0.0;
        }
    // Cholesky L = F F^T in place, the diagonal holding 1 / F_jj (one division per pivot: FP64
    // division is a long instruction sequence on this GPU), then F F^T y = r
    for (int j = 0; j < m; ++j) {
        double d = L[at(j, j)];
        for (int t = 0; t < j; ++t) d -= L[at(j, t)] * L[at(j, t)];
        if (!(d > 0.0)) {
            atomicExch(err_flag, 1);
            return;
        }
        const double rf = 1.0 / sqrt(d);
        L[at(j, j)] = rf;
        for (int a = j + 1; a < m; ++a) {
            double v = L[at(a, j)];
            for (int t = 0; t < j; ++t) v -= L[at(a, t)] * L[at(j, t)];
            L[at(a, j)] = v * rf;
        }
    }
    for (int a = 0; a < m; ++a) {
        double v = y[a];
        for (int t = 0; t < a; ++t) v -= L[at(a, t)] * y[t];
        y[a] = v * L[at(a, a)];
    }
    for (int a = m - 1; a >= 0; --a) {
        double v = y[a];
        for (int t = a + 1; t < m; ++t) v -= L[at(t, a)] * y[t];
        y[a] = v * L[at(a, a)];
    }
    for (int q = q0; q < q1; ++q) {
        const int a = ea[q], b = eb[q];
        double p = Pval[q];
        if (a) p += a > 0 ? y[a - 1] : -y[-a - 1];
        if (b) p += b > 0 ? y[b - 1] : -y[-b - 1];
        Pval[q] = p;
        PTval[pt_pos[q]] = p;
    }
}

template <int M>
void commute_launch(int count, const int32_t* order, const int32_t* rows, const int32_t* Pptr, double* Pval,
                    double* PTval, const int32_t* pt_pos, const int16_t* ea, const int16_t* eb,
                    const int32_t* node_ptr, const double* t, const int32_t* comp, int* err_flag, cudaStream_t s) {
    if (count == 0) return;
    constexpr int T = commute_threads(M);
    const size_t shm = sizeof(double) * (size_t)T * commute_slice(M);
    AMGH_CUDA(cudaFuncSetAttribute(commute_rows_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    commute_rows_kernel<M><<<(count + T - 1) / T, T, shm, s>>>(count, order, rows, Pptr, Pval, PTval, pt_pos, ea, eb,
                                                               node_ptr, t, comp, err_flag);
    AMGH_LAUNCHED();
}

}  // namespace

int commute_size_classes(int* sizes) {
    for (int c = 0; c < 5; ++c) sizes[c] = COMMUTE_SIZES[c];
    return 5;
}

void launch_commute_rows(const int32_t* class_ptr, const int32_t* order, const int32_t* rows, const int32_t* Pptr,
                         double* Pval, double* PTval, const int32_t* pt_pos, const int16_t* ea, const int16_t* eb,
                         const int32_t* node_ptr, const double* t, const int32_t* comp, int* err_flag,
                         cudaStream_t s) {
    commute_launch<8>(class_ptr[1] - class_ptr[0], order + class_ptr[0], rows, Pptr, Pval, PTval, pt_pos, ea, eb,
                      node_ptr, t, comp, err_flag, s);
    commute_launch<16>(class_ptr[2] - class_ptr[1], order + class_ptr[1], rows, Pptr, Pval, PTval, pt_pos, ea, eb,
                       node_ptr, t, comp, err_flag, s);
    commute_launch<32>(class_ptr[3] - class_ptr[2], order + class_ptr[2], rows, Pptr, Pval, PTval, pt_pos, ea, eb,
                       node_ptr, t, comp, err_flag, s);
    commute_launch<64>(class_ptr[4] - class_ptr[3], order + class_ptr[3], rows, Pptr, Pval, PTval, pt_pos, ea, eb,
                       node_ptr, t, comp, err_flag, s);
    commute_launch<128>(class_ptr[5] - class_ptr[4], order + class_ptr[4], rows, Pptr, Pval, PTval, pt_pos, ea, eb,
                        node_ptr, t, comp, err_flag, s);
}

// Symbolic sparse product Z = X Y, one CTA per row of Z: the candidate columns (Y's rows selected
// by the row of X) go into a shared-memory hash set; the count pass writes each row's number of
// distinct columns, the fill pass writes them in ascending order (each key's rank is the number of
// smaller keys), so the pattern does not depend on the order of insertion.  A row whose distinct
// columns exceed the set's load limit raises *overflow and is left to the caller.
constexpr int SYM_THREADS = 256, SYM_SLOTS = 4096, SYM_LIMIT = 3 * SYM_SLOTS / 4;

template <bool FILL>
__global__ void __launch_bounds__(SYM_THREADS) spgemm_symbolic_kernel(
    int nrows, const int32_t* __restrict__ Xptr, const int32_t* __restrict__ Xidx, const int32_t* __restrict__ Yptr,
    const int32_t* __restrict__ Yidx, int32_t* __restrict__ len, const int32_t* __restrict__ Zptr,
    int32_t* __restrict__ Zidx, int* overflow) {
    __shared__ int32_t tab[SYM_SLOTS];
    __shared__ int32_t keys[SYM_LIMIT];
    __shared__ int nkeys, full;
    const int r = blockIdx.x;
    if (r >= nrows) return;
    for (int q = threadIdx.x; q < SYM_SLOTS; q += SYM_THREADS) tab[q] = -1;
    if (threadIdx.x == 0) {
        nkeys = 0;
        full = 0;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = Xptr[r] + warp; t < Xptr[r + 1]; t += SYM_THREADS / 32) {
        const int y = Xidx[t];
        for (int u = Yptr[y] + lane; u < Yptr[y + 1]; u += 32) {
            const int32_t k = Yidx[u];
            uint32_t hsh = ((uint32_t)k * 2654435761u) & (SYM_SLOTS - 1);
            for (int probe = 0; probe < SYM_SLOTS; ++probe) {
                const int32_t old = atomicCAS(&tab[hsh], -1, k);
                if (old == k) break;
                if (old == -1) {
                    const int slot = atomicAdd(&nkeys, 1);
                    if (slot < SYM_LIMIT) keys[slot] = k;
                    else full = 1;
                    break;
                }
                hsh = (hsh + 1) & (SYM_SLOTS - 1);
            }
        }
    }
    __syncthreads();
    if (full) {
        if (threadIdx.x == 0) {
            atomicExch(overflow, 1);
            if (!FILL) len[r] = 0;
        }
        return;
    }
    const int m = nkeys;
    if (!FILL) {
        if (threadIdx.x == 0) len[r] = m;
        return;
    }
    int32_t* out = Zidx + Zptr[r];
    for (int i = threadIdx.x; i < m; i += SYM_THREADS) {
        const int32_t k = keys[i];
        int rank = 0;
        for (int j = 0; j < m; ++j) rank += keys[j] < k;
        out[rank] = k;
    }
}

// Z = X Y symbolically on the device: Z.ptr, Z.idx filled and Z.val allocated.  Returns false (and
// leaves Z empty) when a row has more distinct columns than the shared-memory set holds.
bool spgemm_symbolic(const DevCSR& X, const DevCSR& Y, DevCSR& Z, int* flag, cudaStream_t s) {
    const int n = X.nrows;
    Z.nrows = n;
    Z.ncols = Y.ncols;
    DevArray<int32_t> len;
    len.alloc(std::max(1, n));
    AMGH_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
    if (n > 0) {
        spgemm_symbolic_kernel<false><<<n, SYM_THREADS, 0, s>>>(n, X.ptr.p, X.idx.p, Y.ptr.p, Y.idx.p, len.p, nullptr,
                                                               nullptr, flag);
        AMGH_LAUNCHED();
    }
    std::vector<int32_t> hl(n);
    int of = 0;
    if (n > 0) AMGH_CUDA(cudaMemcpyAsync(hl.data(), len.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    AMGH_CUDA(cudaMemcpyAsync(&of, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGH_CUDA(cudaStreamSynchronize(s));
    if (of) return false;
    std::vector<int32_t> ptr(n + 1, 0);
    int64_t tot = 0;
    for (int r = 0; r < n; ++r) {
        tot += hl[r];
        if (tot >= INT32_MAX) return false;
        ptr[r + 1] = (int32_t)tot;
    }
    Z.nnz = tot;
    Z.max_row = n > 0 ? *std::max_element(hl.begin(), hl.end()) : 0;
    Z.ptr.upload(ptr, s);
    Z.idx.alloc(std::max<int64_t>(1, tot));
    Z.val.alloc(std::max<int64_t>(1, tot));
    if (n > 0) {
        spgemm_symbolic_kernel<true><<<n, SYM_THREADS, 0, s>>>(n, X.ptr.p, X.idx.p, Y.ptr.p, Y.idx.p, nullptr, Z.ptr.p,
                                                              Z.idx.p, flag);
        AMGH_LAUNCHED();
    }
    return true;
}

void launch_ap_numeric(const DevCSR& A, const DevCSR& P, DevCSR& AP, cudaStream_t s) {
    const int n = AP.nrows;
    if (n == 0) return;
    if (AP.max_row > 0 && AP.max_row <= ROWACC_MAX) {
        // warps per CTA so that every warp's output row (columns and sums) fits in shared memory
        const int stride = (AP.max_row + 1) & ~1;
        const size_t per_warp = (size_t)stride * 12;
        const int nw = (int)std::max<size_t>(1, std::min<size_t>(8, (size_t)(96 * 1024) / per_warp));
        const size_t shm = per_warp * nw;
        AMGH_CUDA(cudaFuncSetAttribute(ap_rowacc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        ap_rowacc_kernel<<<(n + nw - 1) / nw, 32 * nw, shm, s>>>(n, A.ptr.p, A.idx.p, A.val.p, P.ptr.p, P.idx.p,
                                                                   P.val.p, AP.ptr.p, AP.idx.p, AP.val.p, stride);
        AMGH_LAUNCHED();
        return;
    }
    const int threads = 256, warps_per_block = threads / 32;
    ap_kernel<<<(n + warps_per_block - 1) / warps_per_block, threads, 0, s>>>(
        n, A.ptr.p, A.idx.p, A.val.p, P.ptr.p, P.idx.p, P.val.p, AP.ptr.p, AP.idx.p, AP.val.p);
    AMGH_LAUNCHED();
}

void launch_ac_numeric(const DevCSR& PT, const DevCSR& AP, DevCSR& Ac, cudaStream_t s) {
    // same kernel shape: row I of Ac = sum_i PT(I, i) AP(i, :)
    launch_ap_numeric(PT, AP, Ac, s);
}

template <class T>
void launch_l1inv(const DevCSR& A, T* out, cudaStream_t s) {
    if (A.nrows == 0) return;
    DevArray<double> tmp;
    double* dst = nullptr;
    if constexpr (std::is_same<T, double>::value) dst = out;
    else { tmp.alloc(A.nrows); dst = tmp.p; }
    l1inv_kernel_d<<<(A.nrows + 255) / 256, 256, 0, s>>>(A.nrows, A.ptr.p, A.val.p, dst);
    AMGH_LAUNCHED();
    if constexpr (!std::is_same<T, double>::value) {
        launch_convert<T>(dst, out, A.nrows, s);
        AMGH_CUDA(cudaStreamSynchronize(s));
    }
}

template <class V>
void launch_sell_fill(const DevCSR& M, Sell<V>& S, cudaStream_t s) {
    if (S.nslices == 0) return;
    sell_fill_kernel<V><<<S.nslices, 32, 0, s>>>(M.nrows, M.ptr.p, M.idx.p, M.val.p, S.nslices, S.slice_ptr.p,
                                                 S.col.p, S.val.p);
    AMGH_LAUNCHED();
}

void launch_coarse_inverse(const DevCSR& A, double* inv, double* work, int* err_flag, cudaStream_t s) {
    coarse_inverse_kernel<<<1, 1024, 0, s>>>(A.nrows, A.ptr.p, A.idx.p, A.val.p, inv, work, err_flag);
    AMGH_LAUNCHED();
}

template <class T>
void launch_convert(const double* in, T* out, int64_t n, cudaStream_t s) {
    if (n == 0) return;
    convert_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
    AMGH_LAUNCHED();
}

#define INST_V(V) template void launch_convert<V>(const double*, V*, int64_t, cudaStream_t);
INST_V(double)
INST_V(float)
INST_V(__nv_bfloat16)
template void launch_sell_fill<double>(const DevCSR&, Sell<double>&, cudaStream_t);
template void launch_l1inv<double>(const DevCSR&, double*, cudaStream_t);
template void launch_l1inv<float>(const DevCSR&, float*, cudaStream_t);

}  // namespace amgh
