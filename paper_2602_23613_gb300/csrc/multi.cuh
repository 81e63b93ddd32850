// Multi-right-hand-side V-cycle and Krylov solver: K systems with the same matrix, vectors stored
// row-major (n x Kp, Kp = K rounded up to a multiple of 32), one matrix read per step for all K.
#pragma once
#include "common.cuh"

namespace amgh {

constexpr int MR_WARPS = 8;   // warps per CTA in the multi-RHS kernels

// per-level data of the multi-RHS engine (CSR patterns and FP64 values shared with the setup; an
// FP32 level adds FP32 copies of the values, inverses and l1 diagonal, and keeps FP32 vectors)
struct MultiLevel {
    int n = 0, ncolours = 0, bmax = 1;
    bool f32 = false;
    const DevCSR* A = nullptr;
    const DevCSR* P = nullptr;    // n x n_c
    const DevCSR* PT = nullptr;   // n_c x n
    std::vector<int32_t> colour_star_begin;   // host, ncolours + 1 (into star_list)
    DevArray<int32_t> star_list;              // stars ordered by colour, ascending within a colour
    DevArray<int32_t> star_ptr, star_idx;     // rows of every star
    DevArray<int64_t> inv_off;                // offset of star j's b x b inverse (row-major)
    DevArray<double> inv;
    DevArray<double> l1inv;
    DevArray<double> F, X, Y, R;              // n x Kp
    // split-K colour steps (levels with long rows): the rows of each colour's stars in order, with
    // their star, position in the star and the star's first position in the colour's list
    bool splitk = false;
    int max_colour_rows = 0;
    std::vector<int32_t> colour_row_begin;    // host, ncolours + 1 (into crow)
    DevArray<int32_t> crow, cstar, cq, cbase;
    DevArray<double> Rc;                      // max_colour_rows x Kp
    DevArray<float> Af, Pf, PTf, invf, l1invf;   // FP32 level: value copies (patterns of A, P, P^T)
    DevArray<float> Ff, Xf, Yf, Rf, Rcf;         // FP32 level: vectors
};

// kernels (multi_kernels.cu); KP = padded width, x/y row-major with leading dimension KP
enum MultiMode { MM_AX = 0, MM_RESID = 1, MM_L1 = 2, MM_ADD = 3 };
void launch_spmm(int mode, const DevCSR& M, int KP, const double* X, const double* F, const double* dinv, double* Y,
                 cudaStream_t s);
// the same on raw arrays: Y (TY) from M (values V) and X (TX); FP64 accumulation when either vector
// type is FP64.  Instantiated for (V, TX, TY) in {ddd, fff, ddf, ffd, dfd, fdf}.
template <class V, class TX, class TY>
void launch_spmm_t(int mode, int nrows, const int32_t* ptr, const int32_t* idx, const V* val, int KP, const TX* X,
                   const TY* F, const TY* dinv, TY* Y, cudaStream_t s);
// one colour step of level L in type T (A's values, inverses, split-K scratch Rc, F and X of type T)
template <class T>
void launch_schwarz_multi_t(const MultiLevel& L, const T* Aval, const T* inv, T* Rc, int colour, int KP, const T* F,
                            T* X, cudaStream_t s);
// Y = Ainv X for a dense n x n FP64 inverse (row-major), X and Y of the coarsest level's type
// (FP64 accumulation); instantiated for (TX, TY) = (double, double), (float, float)
template <class TX, class TY>
void launch_dense_apply_multi_t(const double* Ainv, int n, int KP, const TX* X, TY* Y, cudaStream_t s);
// out = (double) in, n values
void launch_widen(const float* in, int64_t n, double* out, cudaStream_t s);
void launch_star_inverse_rowmajor(const DevCSR& A, int nstars, const int32_t* star_ptr, const int32_t* star_idx,
                                  const int64_t* inv_off, double* inv, int* err_flag, cudaStream_t s);
// column-major (n x k, ld n) <-> row-major padded (n x KP)
void launch_to_rowmajor(const double* in, int64_t n, int k, int KP, double* out, cudaStream_t s);
void launch_to_colmajor(const double* in, int64_t n, int k, int KP, double* out, cudaStream_t s);
// per-column dot products sum_i a[i,c] b[i,c] -> out[c] (deterministic two-stage)
void launch_coldot(const double* a, const double* b, int64_t n, int KP, double* partial, double* out, cudaStream_t s);
// block-CG vector updates with per-column scalars and an active mask
void launch_mcg_update(int64_t n, int KP, double* X, double* R, double* Rold, const double* P, const double* Q,
                       const double* alpha, cudaStream_t s);
void launch_mp_update(int64_t n, int KP, double* P, const double* Z, const double* beta, cudaStream_t s);

}  // namespace amgh
