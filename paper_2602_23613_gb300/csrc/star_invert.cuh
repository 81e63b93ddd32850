// Dense inverse of one SPD smoother block (a node star of at most 32 rows), one warp per block.
#pragma once
#include <cstdint>

namespace amgh {
namespace {

__device__ __forceinline__ int bsearch_i32(const int32_t* a, int lo, int hi, int key) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int v = a[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid;
    }
    return -1;
}

// gather A_BB into M (b x b, row stride S) and invert it by Gauss-Jordan (SPD: no pivoting) into
// I; one warp per star (b <= min(32, S)).  Returns false (on every lane) if a pivot was not
// positive.  The stride only sets the shared-memory footprint: the arithmetic is the same.
template <int S>
__device__ __forceinline__ bool star_invert_s(const int32_t* __restrict__ Aptr, const int32_t* __restrict__ Aidx,
                                              const double* __restrict__ Aval, const int32_t* __restrict__ sidx,
                                              int b0, int b, double* M, double* I, double* fac) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < b; ++r)
        if (lane < b) { M[r * S + lane] = 0.0; I[r * S + lane] = (r == lane); }
    __syncwarp();
    if (lane < b) {
        const int g = sidx[b0 + lane];
        for (int q = Aptr[g]; q < Aptr[g + 1]; ++q) {
            const int c = bsearch_i32(sidx, b0, b0 + b, Aidx[q]);
            if (c >= 0) M[lane * S + (c - b0)] = Aval[q];
        }
    }
    __syncwarp();
    bool ok = true;
    for (int k = 0; k < b; ++k) {
        double piv = M[k * S + k];
        if (!(piv > 0.0)) { ok = false; piv = 1.0; }
        __syncwarp();
        if (lane < b) { M[k * S + lane] /= piv; I[k * S + lane] /= piv; }
        if (lane < b) fac[lane] = M[lane * S + k];
        __syncwarp();
        if (lane < b)
            for (int i = 0; i < b; ++i) {
                if (i == k) continue;
                const double fi = fac[i];
                M[i * S + lane] -= fi * M[k * S + lane];
                I[i * S + lane] -= fi * I[k * S + lane];
            }
        __syncwarp();
    }
    return ok;
}

// gather A_BB into M (b x b, stride 33) and invert it by Gauss-Jordan (SPD: no pivoting) into I;
// one warp per star.  Returns false (on every lane) if a pivot was not positive.
__device__ __noinline__ bool star_invert(const int32_t* __restrict__ Aptr, const int32_t* __restrict__ Aidx,
                            const double* __restrict__ Aval, const int32_t* __restrict__ sidx, int b0, int b,
                            double* M, double* I, double* fac) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < b; ++r)
        if (lane < b) { M[r * 33 + lane] = 0.0; I[r * 33 + lane] = (r == lane); }
    __syncwarp();
    if (lane < b) {
        const int g = sidx[b0 + lane];
        for (int q = Aptr[g]; q < Aptr[g + 1]; ++q) {
            const int c = bsearch_i32(sidx, b0, b0 + b, Aidx[q]);
            if (c >= 0) M[lane * 33 + (c - b0)] = Aval[q];
        }
    }
    __syncwarp();
    bool ok = true;
    for (int k = 0; k < b; ++k) {
        double piv = M[k * 33 + k];
        if (!(piv > 0.0)) { ok = false; piv = 1.0; }
        __syncwarp();
        if (lane < b) { M[k * 33 + lane] /= piv; I[k * 33 + lane] /= piv; }
        if (lane < b) fac[lane] = M[lane * 33 + k];
        __syncwarp();
        if (lane < b)
            for (int i = 0; i < b; ++i) {
                if (i == k) continue;
                const double fi = fac[i];
                M[i * 33 + lane] -= fi * M[k * 33 + lane];
                I[i * 33 + lane] -= fi * I[k * 33 + lane];
            }
        __syncwarp();
    }
    return ok;
}


}  // namespace
}  // namespace amgh
