/*
 * amgh: GB300 (sm_103a) library for the fully algebraic H(curl) algebraic multigrid of
 * Shen, Brannick, Falgout, Kahl, Schroder, "Nodal Coarsening and Sparse Ideal Interpolation for
 * H(curl) Problems in Algebraic Multigrid".
 *
 * Problem (Section 2, Eq. curl): the SPD edge-element system A u = f with A = A^s(mu) + beta A^m,
 * and the discrete gradient G (signed node incidence, de Rham: ker A^s = range G, Eq. deRham).
 * The setup needs only A and G (Section 4): augmentG (Alg. 1), nodal coarsening of the dual
 * operator G~^T A G~ (Alg. 2), matching of fine edges into coarse edges along distance-two
 * nodal paths (Alg. 3), sparse ideal interpolation P_app by interior harmonic extension
 * (Eq. sparseP), G_c = R G I_C (Eq. Gc) and the Galerkin operator A_c = P^T A P (Eq. tl),
 * recursively.  The solve (Section 5) is a V-cycle with one pre- and one post-step of the OSS-l1
 * smoother (symmetrised multiplicative Schwarz on node-star blocks, then l1-Jacobi), used alone or
 * as the preconditioner of conjugate gradients to a relative residual tolerance.
 *
 * Conventions for every entry point:
 *  - Indices are 0-based int32; matrices are CSR with strictly ascending columns in each row.
 *  - "device pointer" means memory of the GPU the handle was created on; "host pointer" means
 *    ordinary or pinned host memory.  Where an argument may be either, the library detects the
 *    kind with cudaPointerGetAttributes and copies host data through its own device buffers.
 *  - All work is enqueued on the handle's stream: amgh_params.stream, or when that is NULL a
 *    blocking stream the handle creates (ordered with the legacy default stream); an entry point
 *    returns after the work it enqueued has completed.
 *  - Every entry point returns an amgh_status and never aborts the process; amgh_last_error()
 *    gives a one-line message for the last failure of the handle (or of a failed setup when the
 *    handle argument is NULL).  After AMGH_ERR_CUDA the handle should be destroyed.
 *  - The handle owns all device memory it allocates (cudaMalloc at setup); the caller owns every
 *    buffer it passes in.  Handles are not thread-safe: use one handle per host thread.
 */
#ifndef AMGH_H
#define AMGH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AMGH_OK = 0,
    AMGH_ERR_INVALID_ARG = 1,   /* malformed input or argument out of range                    */
    AMGH_ERR_NOT_SPD = 2,       /* a Cholesky factorisation met a non-positive pivot            */
    AMGH_ERR_NOT_CONVERGED = 3, /* the solver reached maxit before the tolerance                */
    AMGH_ERR_CUDA = 4,          /* a CUDA runtime call failed                                   */
    AMGH_ERR_OOM = 5,           /* device or host allocation failed                             */
    AMGH_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up                           */
    AMGH_ERR_SETUP_STALL = 7,   /* the finest level produced no coarse edge                     */
    AMGH_ERR_UNSUPPORTED = 8    /* valid input outside the library's limits (e.g. block size)  */
} amgh_status;

typedef struct amgh_ctx* amgh_handle;
typedef struct amgh_mlp_ctx* amgh_mlp;

/* A CSR matrix: nrows x ncols, nnz stored entries.  row_ptr has nrows+1 entries with
 * row_ptr[0] = 0 and row_ptr[nrows] = nnz; col and val have nnz entries.  on_device = 1 when the
 * three arrays are device pointers, 0 when they are host pointers. */
typedef struct {
    int64_t nrows, ncols, nnz;
    const int32_t* row_ptr;
    const int32_t* col;
    const double* val;
    int on_device;
} amgh_csr;

/* storage precision of the V-cycle (hierarchy matrices, interpolation, block inverses, l1
 * diagonal and V-cycle vectors); FP64 keeps everything in double, F32 stores float and
 * accumulates in float, BF16 stores bfloat16 values and accumulates in float. */
enum { AMGH_F64 = 0, AMGH_F32 = 1, AMGH_BF16 = 2 };

/* interior extension of the coarse variables (Eq. sparseP): exact local solves on each coarse
 * edge's patch, or, on the finest level, the values predicted by a trained network (amgh_mlp_*)
 * on the same pattern.  A learned setup measures the convergence factor rho of 10 stand-alone
 * V-cycles on A x = 0 (x0 ~ U(-1,1), SplitMix64 stream 8, seed 0) and falls back to the exact
 * local solves when rho exceeds 1.1 times the exact solves' factor (params.rho_ref, or measured
 * on an exact setup); amgh_info reports which interpolation was kept. */
enum { AMGH_INTERP_LOCAL = 0, AMGH_INTERP_LEARNED = 1, AMGH_INTERP_GEOMETRIC = 2, AMGH_INTERP_CONSTRAINED = 3 };

/* coarse variables: ALGEBRAIC (Section 4: Alg. 1-3 on the nodal dual operator, the default) or
 * REFINEMENT (Section 3, "Ref"): A and G must be the lowest-order Nedelec system of the structured
 * hex mesh of the unit cube with params.mesh_n intervals per side (interior edges numbered x, y,
 * z, each lexicographic by start node with the x index fastest, oriented +axis; interior nodes
 * lexicographic; boundary edges and nodes eliminated), and each coarse edge of the (mesh_n/2)^3
 * mesh pairs its two fine halves with signs (+1, +1); the coarse edges take the coarse mesh's own
 * numbering, so every coarse level is again such a mesh, halved while mesh_n stays even.  With
 * REFINEMENT, interp may also be AMGH_INTERP_GEOMETRIC ("Geo", the comparison of Section 5): the
 * geometric Nedelec interpolation of the coarse mesh, scaled so that its rows on the halves are
 * R^T (a fine edge parallel to its coarse edge one fine step across takes 1/2, two steps 1/4),
 * in place of the local harmonic extensions.
 *
 * AMGH_INTERP_CONSTRAINED (either coarsening) corrects the local extensions to satisfy the
 * commuting relation of Section 2 (Eq. commuting), P G_c = 2 G P_n, which the exact P_app keeps up
 * to O(beta) (Thm. 3.3) and local patches in 3-D lose; the paper leaves a 3-D localisation open, so
 * this is an extension beyond it.  P_n is a nodal interpolation built from the splitting: coarse
 * nodes injected, the middle node of each pair half of each coarse end, every other node the mean
 * of its neighbours in the previous breadth-first layer and of its boundary edges (zero); on a hex
 * refinement that is trilinear interpolation.  The exterior rows R^T satisfy the relation as they
 * are; every interior row of P moves, on its own pattern, to the nearest row (Euclidean) that
 * satisfies its row of the relation, in least squares where none does.  The pattern of P, and so
 * the cost of a V-cycle, is unchanged.  It pays for smooth or piecewise-constant coefficients;
 * where the curl coefficient varies over many decades from element to element it can take more
 * iterations than the plain extension. */
enum { AMGH_COARSEN_ALGEBRAIC = 0, AMGH_COARSEN_REFINEMENT = 1 };

typedef struct {
    int max_levels;       /* at most this many levels, finest included (Section 5: 20)          */
    int coarse_size;      /* stop coarsening once a level has <= coarse_size DoFs (Sec. 5: 32)  */
    int precision;        /* AMGH_F64 | AMGH_F32 | AMGH_BF16: requested V-cycle storage; a level
                             keeps FP64 unless kappa * u <= 1/4 for the largest 1-norm condition
                             estimate kappa of its smoother blocks and the unit roundoff u of the
                             reduced format (BF16 falls back to FP32 first)                     */
    int interp;           /* AMGH_INTERP_LOCAL | AMGH_INTERP_LEARNED | AMGH_INTERP_GEOMETRIC |
                             AMGH_INTERP_CONSTRAINED                                            */
    int ring;             /* rings of interior A-neighbours in a truncated patch (>= 1)        */
    int p_max;            /* largest patch of one local harmonic extension (<= 256)            */
    double theta;         /* strength-of-connection threshold of the nodal C/F split (0.25)    */
    double stall_ratio;   /* stop when n_coarse > stall_ratio * n (0.9)                         */
    void* stream;         /* cudaStream_t for all work of the handle; NULL = a private stream   */
    int dense_tail;       /* the V-cycle's sub-cycle below the first coarse level (not the
                             finest) with at most this many DoFs is linear in its right-hand
                             side; it is computed once at setup, column block by column block,
                             and applied as one dense FP64 (or FP32) operator.  0 = recurse to
                             the coarsest level every time.  Default 8192, at most 16384.       */
    amgh_mlp mlp;         /* network for AMGH_INTERP_LEARNED (see amgh_mlp_*), else NULL        */
    double rho_ref;       /* reference convergence factor of the exact local solves for the
                             learned fallback test; <= 0: measure it with an exact setup       */
    int fuse_restrict;    /* coarse right-hand side r_c = P^T (f - A y) of Eq. tl computed as
                             P^T f - W y with W = P^T A formed at setup: one pass over the rows
                             of P^T and W, no fine residual.  -1: on the Galerkin levels (all
                             but the finest, whose W is about as large as A), where the
                             autotuner keeps it when it times faster than the residual pass plus
                             the restriction; 0: never, W is not formed (default: on the 64^3
                             checkerboard forming W costs more setup time than the pass saves
                             over a 63-iteration solve); 1: on every level                     */
    int coarsening;       /* AMGH_COARSEN_ALGEBRAIC (default) | AMGH_COARSEN_REFINEMENT        */
    int mesh_n;           /* hex mesh intervals per side, for AMGH_COARSEN_REFINEMENT          */
} amgh_params;

/* Set up nsys independent systems (A[i], G[i]) with the same parameters (params may be NULL for
 * the defaults; a stream in params is shared by all handles, NULL gives each its own), as
 * amgh_setup would one by one: out[i] receives system i's handle.  Up to four setups run at
 * once on their own host threads and streams, so one system's host graph steps overlap another's
 * device work; the host's cores are split between them.  Launch choices not yet tuned in this
 * process are timed while other setups run, so they may differ from a lone setup's (results then
 * agree to rounding, not bitwise).  On any failure every handle is destroyed, out[] is NULL and
 * the status of the first failing system is returned (amgh_last_error(NULL) names it).  The
 * batch counterpart of Section 4's setup for the many-systems workload. */
amgh_status amgh_batch_setup(int nsys, const amgh_csr* A, const amgh_csr* G, const amgh_params* params,
                             amgh_handle* out);

/* Fill *p with the defaults: max_levels 20, coarse_size 100, F64, LOCAL, ring 1, p_max 128,
 * theta 0.25, stall_ratio 0.9, stream NULL, dense_tail 8192, fuse_restrict 0, coarsening ALGEBRAIC,
 * mesh_n 0. */
void amgh_default_params(amgh_params* p);

/* Build the hierarchy for A (n x n, SPD, symmetric pattern) and the discrete gradient G (n x m,
 * every row holds at most two entries equal to +-1, two entries of opposite sign; a row with one
 * entry is an edge touching the eliminated boundary, a row with none an interior edge joining two
 * boundary nodes).  Section 4
 * (Alg. 1-3, Eq. sparseP, Eq. Gc) recursed per Section 5's limits.  A and G are deep-copied; the
 * caller may free them on return.  Errors: INVALID_ARG for malformed CSR, non-square A, a G row
 * with more than 2 entries, an entry other than +-1, or a two-entry row whose entries share a sign;
 * NOT_SPD when a local or coarsest factorisation fails; SETUP_STALL when level 0 has no coarse
 * edge; UNSUPPORTED for a smoother block larger than 32 DoFs or a coarsest level larger than
 * 2048 DoFs. On failure *out is NULL. */
amgh_status amgh_setup(const amgh_csr* A, const amgh_csr* G, const amgh_params* params,
                       amgh_handle* out);

/* Host-only variant of amgh_setup for inspecting the graph steps of the finest level without a
 * GPU: runs Alg. 1-3, the patch construction of Eq. sparseP, the symbolic Galerkin pattern and
 * the smoother stars and colouring of level 0 on the host and makes no CUDA call (A and G must be
 * host CSR).  On the returned handle only amgh_level_structure(h, 0, ...), amgh_level_matrix(h,
 * 0, which) (which = 1 returns P's pattern with the exterior +-1 and zeros elsewhere; which = 3
 * returns the symbolic pattern of P^T A P with zero values; which = 4 the nodal interpolation of
 * the commuting correction when interp is CONSTRAINED), amgh_last_error and amgh_destroy are
 * valid; every other call returns INVALID_ARG.  Errors as amgh_setup. */
amgh_status amgh_setup_host_structure(const amgh_csr* A, const amgh_csr* G, const amgh_params* params,
                                      amgh_handle* out);

/* z = B r, one V-cycle (Eq. tl applied recursively: zero initial guess, OSS-l1 pre-step,
 * residual restriction P^T, coarse correction, prolongation P, OSS-l1 post-step; dense Cholesky
 * on the coarsest level).  r and z: n doubles, host or device pointers (both of the same kind),
 * may not alias. */
amgh_status amgh_vcycle(amgh_handle h, const double* r, double* z);

/* Preconditioned conjugate gradients (Section 5) on the finest A with the V-cycle as the
 * preconditioner.  The loop runs on the device inside one CUDA graph (conditional WHILE node);
 * while kernel timing is enabled (amgh_profile) it is driven from the host instead.  Stops when ||f - A x_k||_2 (as updated by the recurrence) <= tol ||f - A x_0||_2
 * or after maxit iterations.  x holds x_0 on entry and the solution on return; f and x are n
 * doubles, host or device (same kind).  With an FP32/BF16 hierarchy the outer loop is flexible
 * CG (beta = <z_k+1, r_k+1 - r_k> / <z_k, r_k>) with FP64 vectors, SpMV and dots.  iters and
 * relres (may be NULL) receive the iteration count and the final relative residual.
 * Returns NOT_CONVERGED (with x, iters, relres filled) when maxit is reached. */
amgh_status amgh_pcg_solve(amgh_handle h, const double* f, double* x, double tol, int maxit,
                           int* iters, double* relres);

/* Solve nsys independent systems at once.  hs[i] comes from amgh_setup (any sizes and
 * precisions, same GPU); f[i] and x[i] are device pointers of n_i doubles (x[i] holds x0 on entry,
 * the solution on return).  All systems are enqueued as independent branches of one CUDA graph
 * whose branches each run their PCG loop on the device (a conditional WHILE node per system that
 * stops at tol or maxit), and the graph is launched once on hs[0]'s stream; no host round trip
 * happens until every system has stopped.  iters and relres (may be NULL) receive nsys entries.
 * Returns NOT_CONVERGED if any system reached maxit.  Section 5's solver per system. */
amgh_status amgh_batch_pcg_solve(int nsys, const amgh_handle* hs, const double* const* f, double* const* x,
                                 double tol, int maxit, int* iters, double* relres);

/* PCG exactly as amgh_pcg_solve, but allocating nothing: its Krylov buffers (search direction,
 * A times it, previous residual, partial sums, scalars) live in one fixed device array that the
 * library defines at file scope (6.3 MB on every GPU that loads the library, kept until the
 * process exits), the loop is driven from the host and the V-cycle kernels are launched one by
 * one, so no memory, graph or staging buffer is created.  The loop reads its scalars into the
 * handle's pinned host buffer and synchronises the handle's stream once per iteration.  It is
 * meant for callers that cannot allocate device memory when they solve: applications whose
 * caching allocator has reserved nearly all device memory, and loops that cannot afford the
 * device-wide synchronisation that cudaMalloc/cudaFree bring.  The paper has no counterpart; it
 * is a deployment variant.
 *  - f and x must be device pointers on the handle's device, and that device must be current;
 *    otherwise INVALID_ARG.  n <= 262144 rows; larger systems are rejected with INVALID_ARG.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 *    make that first call before any stream capture begins.
 *  - All calls share the array: calls whose work overlaps on the GPU (other host threads, other
 *    handles on other streams) race and must be serialised by the caller.
 * Returns as amgh_pcg_solve. */
amgh_status amgh_pcg_solve_noalloc(amgh_handle h, const double* f, double* x, double tol, int maxit,
                                   int* iters, double* relres);

/* k right-hand sides with the same matrix (Section 5's PCG per column): F and X are n x k
 * column-major (column c at F + c n), host or device (same kind), X holds the initial guesses.
 * The k CG recurrences are independent (their own alpha, beta and stopping test); every matrix
 * product and V-cycle step is done for all unconverged columns at once, reading each matrix
 * entry once per step (sparse matrix times a row-major n x k block).  Each level of this
 * entry's V-cycle has the storage the handle's own V-cycle chose for it (amgh_info precision):
 * FP64, or FP32 values and vectors with FP32 accumulation (BF16 levels run in FP32 here).  With
 * any FP32 level the recurrences are flexible CG (beta = <z_k+1, r_k+1 - r_k> / <z_k, r_k>);
 * the outer vectors, products and dots stay FP64.  iters and relres (may be NULL) receive k
 * entries.  1 <= k <= 4096.  Returns NOT_CONVERGED if any column reached maxit. */
amgh_status amgh_pcg_solve_multi(amgh_handle h, const double* F, double* X, int k, double tol, int maxit,
                                 int* iters, double* relres);

/* Z = B R for k right-hand sides at once (n x k column-major device arrays), with the level
 * storage described for amgh_pcg_solve_multi. */
amgh_status amgh_vcycle_multi(amgh_handle h, const double* R, double* Z, int k);

/* Stand-alone V-cycle iteration x <- x + B (f - A x) (Section 5, "AMG" counts), same stopping
 * rule and argument conventions as amgh_pcg_solve, on the true residual. */
amgh_status amgh_amg_solve(amgh_handle h, const double* f, double* x, double tol, int maxit,
                           int* iters, double* relres);

typedef struct {
    int levels;
    int64_t n[32];        /* DoFs per level                                                    */
    int64_t nnz[32];      /* stored entries of A_l                                             */
    int64_t nnz_p[32];    /* stored entries of P_l (0 on the coarsest level)                   */
    int ncolours[32];     /* smoother colours per level (0 on the coarsest level)             */
    int max_block[32];    /* largest smoother block per level                                  */
    int max_patch[32];    /* largest interpolation patch per level                             */
    double op_complexity; /* sum nnz(A_l) / nnz(A_0)                                           */
    double grid_complexity; /* sum n_l / n_0                                                    */
    double setup_host_ms; /* host graph steps (Alg. 1-3, patterns, colouring)                 */
    double setup_device_ms; /* device numerics (patch solves, Galerkin product, inverses, tuning) */
    int precision[32];    /* storage precision each level ended up with (AMGH_F64/F32/BF16)   */
    int lanes[32];        /* lanes per row of the level's smoother layout (autotuned)          */
    int fused[32];        /* launch mode of the level's Schwarz sweep: 0 one launch per colour
                             step, 1 one single-CTA launch, 2 one cooperative launch with grid
                             barriers, 3 the same with chunks staged in shared memory, 4 one
                             streaming launch per colour step (chunks staged by bulk copies),
                             5 staged chunks in one thread-block cluster (hardware barrier),
                             6 one launch per colour step with programmatic dependent launch,
                             7 one cluster of 512-thread CTAs prefetching each step's matrix
                             entries into registers before the hardware cluster barrier,
                             8 one cluster of 8 or 16 CTAs, each holding the level's x in
                             shared memory (updated rows written to every copy through
                             distributed shared memory), for levels whose x fits in a CTA,
                             9 the same pipelined item walk as one cooperative grid with x in
                             global memory and a counter barrier between colour steps.
                             The autotuner picks the fastest; AMGH_TUNE=0 disables tuning and
                             AMGH_SMOOTHER_MODE=colour|pdl|stream1|stream2|fused|persistent|
                             staged|cluster|cluster2|resident|pipeline restricts it to one
                             mode where the level has it (resident-<C>x<G>-L<lanes>, e.g.
                             resident-16x2-L8: one shape of mode 8 with C CTAs of G 256-thread
                             chunk groups; pipeline-<C>x<G>-L<lanes> likewise for mode 9).     */
    double block_kappa[32]; /* largest 1-norm condition estimate of the level's smoother blocks
                               (coarsest level: of its matrix); estimated only when a reduced
                               precision is requested, else 0 (coarsest level: always)          */
    int dense_tail;       /* level whose sub-cycle is applied as a dense operator, or -1       */
    int interp_used;      /* the interpolation the hierarchy holds (LEARNED only if it passed
                             the fallback test)                                                 */
    double rho;           /* measured convergence factor of the kept hierarchy (learned setups)  */
    double rho_exact;     /* the exact local solves' factor it was compared with               */
    double interp_ms;     /* wall time of filling the finest level's P values (solves or network) */
    int fused_rr[32];     /* 1 where the V-cycle computes the coarse right-hand side in the fused
                             pass over P^T and W = P^T A, 0 where residual and restriction run
                             apart                                                             */
} amgh_hier_info;

/* Hierarchy statistics (levels, sizes, complexities as defined in Section 5, setup time split). */
amgh_status amgh_info(amgh_handle h, amgh_hier_info* info);

/* Structural outputs of the setup on level l (0 <= l < levels-1), into host arrays.  Any pointer
 * may be NULL to skip it; sizes are those reported by the query form: call first with all
 * pointers NULL to obtain the counts.
 *   ncoarse_nodes / cf_state: length n_nodes_aug = columns of G~ (Alg. 1): state 1 = C, 2 = F
 *   coarse_edges: 7 ints per coarse edge in creation order: DoF1, s1, DoF2, s2, i, k, j (Alg. 3)
 *   coarse_nodes: the kept columns of R G (Eq. Gc), ascending
 *   patch_ptr / patch_idx: CSR of the sorted patch of every coarse edge (Eq. sparseP)
 *   colour: smoother colour of every star (one star per column of G_l) */
amgh_status amgh_level_structure(amgh_handle h, int l, int64_t* n_nodes_aug, int64_t* n_edges,
                                 int64_t* n_coarse_nodes, int64_t* patch_nnz, int64_t* n_stars,
                                 int8_t* cf_state, int32_t* coarse_edges, int32_t* coarse_nodes,
                                 int32_t* patch_ptr, int32_t* patch_idx, int32_t* colour);

/* Copy a level matrix to host CSR arrays (FP64 values as computed on the device).
 * which = 0: A_l (n_l x n_l); 1: P_l (n_l x n_{l+1}); 2: G_l (n_l x m_l); 3: the symbolic pattern
 * of P_l^T A_l P_l with the device values of A_{l+1} (zeros on a structure-only handle); 4: the
 * nodal interpolation P_n of Eq. commuting that the commuting correction used on level l (m_l x
 * coarse nodes, host-computed; interp CONSTRAINED only, on a structure-only handle too, else
 * INVALID_ARG).
 * Query form: pass row_ptr = col = val = NULL to receive nrows, ncols, nnz only. */
amgh_status amgh_level_matrix(amgh_handle h, int l, int which, int64_t* nrows, int64_t* ncols,
                              int64_t* nnz, int32_t* row_ptr, int32_t* col, double* val);

/* Single steps of the V-cycle on level l, for testing the kernels one by one.  Device pointers
 * of n_l (or n_{l+1}) doubles.  op = 0: y = A_l x;  1: y = f - A_l x;  2: x <- OSS-l1 pre-step
 * (x in/out, f the right-hand side);  3: x <- OSS-l1 post-step;  4: y = P_l^T x (restriction);
 * 5: y <- y + P_l x (prolongation);  6: y = A_L^{-1} x on the coarsest level L (l ignored);
 * 7: y = P_l^T (f - A_l x) by the fused pass (P_l^T f - W_l x, W_l = P_l^T A_l; Eq. tl), on a
 * level that holds W_l (INVALID_ARG otherwise; params.fuse_restrict = 1 gives every level W). */
amgh_status amgh_level_apply(amgh_handle h, int l, int op, const double* f, const double* x,
                             double* y);

/* Kernel timing, for the roofline: when enabled the library brackets every launch of the
 * kernels of class `kind` on level `level` with CUDA events on its stream.  kind: 0 Schwarz
 * colour sweep, 1 l1-Jacobi, 2 residual, 3 restriction, 4 prolongation, 5 coarsest solve,
 * 6 outer SpMV, 7 fused residual + restriction.  amgh_kernel_stats returns the number of bracketed launches, their summed
 * duration (ms) and the algorithmic bytes they moved (sum over launches of the bytes each launch
 * must read and write once: matrix values and indices, block inverses, vectors). */
amgh_status amgh_profile(amgh_handle h, int enable, int kind, int level);
amgh_status amgh_kernel_stats(amgh_handle h, int64_t* launches, double* total_ms,
                              double* algorithmic_bytes);

/* Number of kernels the library has launched in this process, over all handles (a CUDA-graph
 * replay counts every kernel it runs); the handle argument may be NULL. */
int64_t amgh_launch_count(amgh_handle h);

/* ---- learned interpolation weights (a 3-layer perceptron, width 64, FP32 or BF16 storage,
 * trained on the GPU) ----
 * Input per finest-level coarse edge: 3 features per patch slot (64 slots) plus 2, from A alone
 * (signed log magnitudes, normalised by A[DoF1, DoF1], of the slot's diagonal, of the local
 * right-hand side of Eq. sparseP and of its coupling inside the patch); output: the patch values
 * of the edge's column of P.  Training target: the exact local solves; loss: masked mean squared
 * error; optimiser: Adam. */
amgh_status amgh_mlp_create(uint64_t seed, amgh_mlp* out);   /* Glorot-uniform init, stream 7   */
/* storage of the network's products: AMGH_F32 (the default) or AMGH_BF16, where the inputs, the
 * weight matrices and the hidden activations are held as bfloat16 (nearest, ties to even) and
 * every product accumulates in FP32; biases, outputs, gradients, the Adam state and the master
 * weights (what amgh_mlp_params reads and writes) stay FP32.  Applies to every later prediction,
 * gradient and training step, and to setups that use the network.  INVALID_ARG for any other
 * value. */
amgh_status amgh_mlp_set_precision(amgh_mlp m, int precision);
/* append the finest-level samples (features, exact patch values) of a hierarchy built with exact
 * local solves (patches of at most 64 DoFs) to the network's device-resident training set */
amgh_status amgh_mlp_add_samples(amgh_mlp m, amgh_handle h);
int64_t amgh_mlp_num_samples(amgh_mlp m);
/* epochs over the samples in shuffled batches (Fisher-Yates from stream 7, seed + epoch) */
amgh_status amgh_mlp_train(amgh_mlp m, int epochs, int batch, double lr, uint64_t seed, double* final_loss);
/* parameters W1 (194x64), b1, W2 (64x64), b2, W3 (64x64), b3, row-major FP32, concatenated:
 * copy them out (out != NULL) and/or in (in != NULL); count receives their number */
amgh_status amgh_mlp_params(amgh_mlp m, float* out, float* in, int64_t* count);
/* loss and gradient (same layout as the parameters) of one batch of host arrays X (nb x 194),
 * T and M (nb x 64) */
amgh_status amgh_mlp_loss_grad(amgh_mlp m, const float* X, const float* T, const float* M, int nb, double* loss,
                               float* grad);
amgh_status amgh_mlp_predict(amgh_mlp m, const float* X, int64_t n, float* Y);   /* host arrays */
/* the finest level's features (n x 194), exact targets and masks (n x 64) of a hierarchy, into host
 * arrays (NULL: skip); n receives the number of coarse edges */
amgh_status amgh_mlp_features(amgh_handle h, float* X, float* T, float* M, int64_t* n);
const char* amgh_mlp_last_error(amgh_mlp m);
void amgh_mlp_destroy(amgh_mlp m);

/* Self-test of the device-side bounded waits (the grid barriers of the cooperative smoother
 * sweeps): launches a two-CTA cooperative grid whose barrier expects one arrival more than the
 * grid has, so it can never complete.  Every wait must give up after its bound (about a second),
 * raise the error flag and return; the context stays usable.  Returns AMGH_ERR_TIMEOUT when that
 * happened (the expected outcome), with the elapsed wall time in *seconds; any other status is a
 * failure of the mechanism.  The paper has no counterpart. */
amgh_status amgh_selftest_wait_timeout(double* seconds);

const char* amgh_last_error(amgh_handle h);
void amgh_destroy(amgh_handle h);

#ifdef __cplusplus
}
#endif

#endif /* AMGH_H */
