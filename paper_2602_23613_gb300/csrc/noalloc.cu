// Allocation-free PCG solve: the Krylov buffers live in a fixed file-scope device array instead
// of memory the library would allocate.  For callers that cannot allocate device memory at solve
// time: applications whose caching allocator has reserved nearly all device memory, and loops
// that cannot afford the device-wide synchronisation that cudaMalloc/cudaFree bring.
#include <mutex>
#include <string>

#include "kernels.h"
#include "krylov_scratch.h"

namespace amgh {

namespace {

constexpr int64_t NOALLOC_MAX_ROWS = 262144;
constexpr size_t NOALLOC_DOUBLES = 3 * (size_t)NOALLOC_MAX_ROWS + 2 * (size_t)RED_BLOCKS + 16;

// One copy per GPU that loads the library (6.3 MB), held until the process exits.  Every call
// shares it, so calls whose work overlaps on the GPU race with each other.
static __device__ __align__(256) double g_krylov_scratch[NOALLOC_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once per device (the host
// symbol is only a stand-in and must never be handed to a kernel).
amgh_status scratch_on_current_device(double** out, const char** msg) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        *msg = "no usable current CUDA device";
        return AMGH_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_krylov_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            *msg = "cudaGetSymbolAddress of the Krylov scratch array failed";
            return AMGH_ERR_CUDA;
        }
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return AMGH_OK;
}

}  // namespace

}  // namespace amgh

extern "C" amgh_status amgh_pcg_solve_noalloc(amgh_handle h, const double* f, double* x, double tol, int maxit,
                                              int* iters, double* relres) {
    using namespace amgh;
    if (!h) return AMGH_ERR_INVALID_ARG;
    double* base = nullptr;
    const char* msg = nullptr;
    const amgh_status st = scratch_on_current_device(&base, &msg);
    if (st != AMGH_OK) return fail_with(h, st, msg);
    KrylovScratch ks;
    ks.p = base;
    ks.q = base + NOALLOC_MAX_ROWS;
    ks.r_old = base + 2 * NOALLOC_MAX_ROWS;
    ks.partial = base + 3 * NOALLOC_MAX_ROWS;
    ks.scal = ks.partial + 2 * RED_BLOCKS;
    return pcg_with_scratch(h, f, x, tol, maxit, iters, relres, ks, NOALLOC_MAX_ROWS);
}
