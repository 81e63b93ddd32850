// Launchers of the V-cycle kernels with L lanes per row and per-level precisions.
#pragma once
#include "layout.h"

namespace amgh {

enum SellModeL { SM_AX = 0, SM_RESID = 1, SM_L1 = 2, SM_ADD = 3 };

// MODE AX: y = M x;  RESID: y = f - M x;  L1: y = x + dinv (f - M x);  ADD: y += M x.
// V: storage of M; TX: type of x; TY: type of f, dinv and y.  Accumulation in double when either
// vector type is double, else in float.  Supported L: 1, 2, 4, 8, 16, 32.
template <class V, class TX, class TY>
void launch_sellL(int mode, const SellL<V>& M, const TX* x, const TY* f, const TY* dinv, TY* y, cudaStream_t s);

// fused residual and restriction: out = PT f - W y with W = P^T A (so out = P^T (f - A y)), one
// pass over the rows of PT and W, which must share L and the row count.  V: storage of both;
// TX: type of f and y; TY: type of out; accumulation as in launch_sellL.
template <class V, class TX, class TY>
void launch_rr(const SellL<V>& PT, const SellL<V>& W, const TX* f, const TX* y, TY* out, cudaStream_t s);

// one colour of the multiplicative Schwarz sweep (chunks [cta_begin, cta_end) of the colour); with
// S.stream_grid > 0 as a streaming launch of at most that many CTAs
template <class V, class T>
void launch_schwarz_colourL(const SmootherL<V>& S, int colour, const T* f, T* x, cudaStream_t s);
// whole symmetric sweep (colours 0..C-1, C-2..0) in one single-CTA launch
template <class V, class T>
void launch_schwarz_fused(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s);

// whole symmetric sweep in one cooperative launch of S.persist CTAs (grid barriers between colours;
// a barrier wait that gives up sets *S.wait_err and the sweep ends early)
template <class V, class T>
void launch_schwarz_persistent(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s);
// largest grid of the persistent sweep that is co-resident on this device for L lanes per row
template <class V, class T>
int schwarz_persistent_cap(int L);
// largest co-resident grid of the staged persistent sweep (chunks staged in shared memory by
// bulk async copies; needs S.wmax), 0 when its two stage buffers do not fit
template <class V, class T>
int schwarz_staged_cap(const SmootherL<V>& S);
// largest co-resident grid of the streaming colour step (chunks staged in shared memory by bulk
// async copies, nbuf = 1 or 2 buffers per CTA; S.stream_grid > 0 selects it), 0 when it cannot
// run for this smoother
template <class V, class T>
int schwarz_stream_cap(const SmootherL<V>& S, int nbuf);
// whether the staged sweep can run as one thread-block cluster of `size` CTAs (S.persist = size,
// S.staged and S.cluster then select it): colour steps ordered by the hardware cluster barrier
template <class V, class T>
bool schwarz_cluster_ok(const SmootherL<V>& S, int size);
// self-test: a grid barrier that can never complete (one arrival short) must give up after its
// bounded wait and raise *err; returns whether it did (err: device int)
bool run_wait_timeout_probe(int* err, cudaStream_t s);
// whether the register-prefetching sweep can run as one cluster of `size` 512-thread CTAs (two
// chunk groups each: colours of at most 2 x size chunks; S.cluster2 = size selects it)
template <class V, class T>
bool schwarz_cluster2_ok(const SmootherL<V>& S, int size);
// whether the resident sweep can run as one cluster of `size` CTAs of `groups` x 256 threads:
// every CTA holds x (S.n values of T) in shared memory; L = 4, 8, 16 or 32.  Raises the kernel's
// shared-memory and cluster-size limits.  S.resident = size, S.resident_g = groups select it.
template <class V, class T>
bool schwarz_resident_ok(const SmootherL<V>& S, int size, int groups);
// co-resident CTAs of the pipelined grid sweep (the resident sweep's item walk over a cooperative
// grid, x in global memory, counter barrier; S.resident = grid, S.resident_grid select it), 0
// when L is not 4, 8, 16 or 32
template <class V, class T>
int schwarz_pipeline_cap(const SmootherL<V>& S, int groups);
// host-built item lists of the resident sweep for that shape (kept until the shape changes)
template <class V>
void schwarz_resident_prepare(SmootherL<V>& S, int size, int groups, cudaStream_t s);
// whole symmetric sweep with x resident in the shared memory of one thread-block cluster
template <class V, class T>
void launch_schwarz_resident(const SmootherL<V>& S, const T* f, T* x, cudaStream_t s);
// whether a cooperative launch can be captured into a graph and replayed on the current device
bool cooperative_capture_works();

// setup: fill the SELL-L copy of a CSR matrix, the smoother's slot rows, and the star inverses
template <class V>
void launch_sellL_fill(const DevCSR& M, SellL<V>& S, cudaStream_t s);
template <class V>
void launch_slotL_fill(const DevCSR& A, SmootherL<V>& S, cudaStream_t s);
template <class V>
void launch_star_inverseL(const DevCSR& A, int nstars, const int32_t* star_ptr, const int32_t* star_idx,
                          const int32_t* star_cta, const int32_t* star_base, SmootherL<V>& S, int* err_flag,
                          cudaStream_t s);
// largest 1-norm condition estimate ||A_BB||_1 ||A_BB^-1||_1 over the stars (FP64), into *kappa
// (device double, must be zeroed by the caller)
void launch_star_kappa(const DevCSR& A, int nstars, const int32_t* star_ptr, const int32_t* star_idx,
                       double* kappa, int* err_flag, cudaStream_t s);

}  // namespace amgh
