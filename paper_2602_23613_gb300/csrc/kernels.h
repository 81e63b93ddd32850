// Launchers of the device kernels (defined in setup_kernels.cu and solve_kernels.cu).
#pragma once
#include "common.cuh"

namespace amgh {

// ---------------- setup numerics (FP64) ----------------------------------------------------
// Local interior harmonic extension (Eq. sparseP): for coarse edge c with exterior pair
// (d1, s1), (d2, s2) and sorted patch p, solve A_pp x = -(A_{p,d1} s1 + A_{p,d2} s2) by dense
// Cholesky and scatter x into P (positions pos_P) and P^T (positions pos_PT).
// exterior values of P and P^T (R^T: s1 at DoF1, s2 at DoF2 of every coarse edge) at the given
// positions; the other entries are left as they are
void launch_ext_scatter(int nc, const int32_t* edges4, const int64_t* ext_P, const int64_t* ext_PT, double* Pval,
                        double* PTval, cudaStream_t s);
void launch_patch_solve(const DevCSR& A, int nc, const int32_t* edges4, const int32_t* patch_ptr,
                        const int32_t* patch_idx, const int64_t* pos_P, const int64_t* pos_PT,
                        double* Pval, double* PTval, int max_patch, int* err_flag, cudaStream_t s);

// Eq. commuting: each listed interior row of P (values after the local solves) moved on its own
// pattern to the nearest row satisfying row i of P G_c = 2 G P_n, from the host-built per-row data
// (see CommutingRows); P^T's copy follows.  Rows go by size class: order[class_ptr[c] ..
// class_ptr[c+1]) lists the rows (indices into rows) with at most sizes[c] local nodes, sizes from
// commute_size_classes (ascending; returns their number, 5).  A non-positive pivot, or a row
// larger than its class, sets *err_flag.  class_ptr is a host array.
int commute_size_classes(int* sizes);
void launch_commute_rows(const int32_t* class_ptr, const int32_t* order, const int32_t* rows, const int32_t* Pptr,
                         double* Pval, double* PTval, const int32_t* pt_pos, const int16_t* ea, const int16_t* eb,
                         const int32_t* node_ptr, const double* t, const int32_t* comp, int* err_flag,
                         cudaStream_t s);

// Galerkin product A_c = P^T (A P) on given symbolic patterns (Eq. tl), FP64, deterministic order.
// symbolic Z = X Y on the device (sorted columns per row); false when a row overflows the
// kernel's shared-memory set (the caller then computes the pattern on the host)
bool spgemm_symbolic(const DevCSR& X, const DevCSR& Y, DevCSR& Z, int* flag, cudaStream_t s);
void launch_ap_numeric(const DevCSR& A, const DevCSR& P, DevCSR& AP, cudaStream_t s);
void launch_ac_numeric(const DevCSR& PT, const DevCSR& AP, DevCSR& Ac, cudaStream_t s);

// l1 row norms: out[i] = 1 / sum_j |a_ij|
template <class T>
void launch_l1inv(const DevCSR& A, T* out, cudaStream_t s);

// SELL copy (one lane per row) of a CSR matrix in storage type V, for the outer FP64 SpMV
template <class V>
void launch_sell_fill(const DevCSR& M, Sell<V>& S, cudaStream_t s);

// Dense inverse of the coarsest matrix (Cholesky factor, then inverse of the factor) into inv
// (n x n, FP64, row-major); work: n*n doubles.
void launch_coarse_inverse(const DevCSR& A, double* inv, double* work, int* err_flag, cudaStream_t s);

template <class T>
void launch_convert(const double* in, T* out, int64_t n, cudaStream_t s);
template <class T>
void launch_to_double(const T* in, double* out, int64_t n, cudaStream_t s);

// ---------------- solve (V-cycle precision V storage, T vectors) ---------------------------
enum SellMode { SELL_AX = 0, SELL_RESID = 1, SELL_L1 = 2, SELL_ADD = 3 };
// outer FP64 SpMV passes.  MODE AX: y = A x; RESID: y = f - A x
template <class V, class T>
void launch_sell(int mode, const Sell<V>& A, const T* x, const T* f, const T* dinv, T* y,
                 cudaStream_t s);

template <class T>
void launch_coarse_apply(const T* inv, int n, const T* x, T* y, cudaStream_t s);

// ---------------- outer Krylov vectors (FP64) ------------------------------------------------
constexpr int RED_BLOCKS = 608;     // 4 x 152 SMs: fixed grid => deterministic reductions
constexpr int RED_THREADS = 256;
// q = A p (SELL FP64) and partial sums of p.q
void launch_spmv_dot(const Sell<double>& A, const double* p, double* q, double* partial, cudaStream_t s);
// final reduction of RED_BLOCKS partials into scal[slot] (+ op on scalars)
enum ScalarOp { SC_STORE = 0, SC_ALPHA = 1, SC_BETA_CG = 2, SC_BETA_FCG = 3, SC_RZ = 4 };
void launch_reduce(const double* partial, int nvals, double* scal, int op, cudaStream_t s);
// x += alpha p, r -= alpha q (alpha = scal[RZ]/scal[PQ]); r_old = r if r_old; partial r.r
void launch_cg_update(int64_t n, double* x, double* r, double* r_old, const double* p, const double* q,
                      const double* scal, double* partial, cudaStream_t s);
// partial sums of r.z (and z.r_old when r_old != nullptr, stored in the second half)
void launch_dot2(int64_t n, const double* r, const double* z, const double* r_old, double* partial,
                 cudaStream_t s);
// p = z + beta p (beta = scal[BETA])
void launch_p_update(int64_t n, double* p, const double* z, const double* scal, cudaStream_t s);
// generic dot partials a.b
void launch_dot(int64_t n, const double* a, const double* b, double* partial, cudaStream_t s);
// x += y
void launch_axpy1(int64_t n, double* x, const double* y, cudaStream_t s);

// indices into the device scalar block of the Krylov loop
enum Scal { S_RZ = 0, S_PQ = 1, S_RR = 2, S_ALPHA = 3, S_BETA = 4, S_RZ_NEW = 5, S_ZROLD = 6, S_TMP = 7,
            S_R0 = 8, S_REL = 9, S_COUNT = 10 };

// device-resident stopping test: iteration count += 1, rel = sqrt(scal[S_TMP]) / scal[S_R0],
// keep looping (WHILE handle = 1) while rel > tol and count < maxit
void launch_pcg_check(cudaGraphConditionalHandle hw, double* scal, int* iter, double tol, int maxit,
                      cudaStream_t s);
// scal[S_R0] = sqrt(scal[S_TMP]); iteration count = 0
void launch_pcg_start(double* scal, int* iter, cudaStream_t s);

}  // namespace amgh
