// Internal interface between the driver and the allocation-free PCG entry point.
#pragma once
#include <cstdint>

#include "../../include/amgh.h"

namespace amgh {

// device buffers of the Krylov loop that the caller provides instead of the handle
struct KrylovScratch {
    double* p;        // search direction, n doubles
    double* q;        // A p, n doubles
    double* r_old;    // previous residual (flexible CG), n doubles
    double* partial;  // 2 x RED_BLOCKS partial sums
    double* scal;     // S_COUNT scalars
};

// records `msg` as the handle's last error and returns `st`
amgh_status fail_with(amgh_handle h, amgh_status st, const char* msg);

// PCG / flexible CG on the handle's finest level with the Krylov buffers in `ks`: host-driven
// loop, eager kernel launches, no allocation.  f and x must be device pointers of n doubles with
// n <= max_rows.
amgh_status pcg_with_scratch(amgh_handle h, const double* f, double* x, double tol, int maxit, int* iters,
                             double* relres, const KrylovScratch& ks, int64_t max_rows);

}  // namespace amgh
