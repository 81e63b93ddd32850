// Internal declarations shared by the CUDA translation units of libamgh.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/amgh.h"
#include "host_graph.h"

namespace amgh {

struct CudaError {
    cudaError_t code;
    std::string where;
};

#define AMGH_CUDA(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) throw ::amgh::CudaError{e_, std::string(#call) + " @" +    \
                                                           std::to_string(__LINE__)};     \
    } while (0)

// kernel launches issued by the library in this process (graph replays add their kernel count)
std::atomic<int64_t>& launch_counter();

#define AMGH_LAUNCHED()                          \
    do {                                         \
        AMGH_CUDA(cudaGetLastError());           \
        ::amgh::launch_counter().fetch_add(1);   \
    } while (0)

// typed device allocation owned by the handle
template <class T>
struct DevArray {
    T* p = nullptr;
    size_t n = 0;
    DevArray() = default;
    DevArray(const DevArray&) = delete;
    DevArray& operator=(const DevArray&) = delete;
    DevArray(DevArray&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DevArray& operator=(DevArray&& o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DevArray() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count) {
        release();
        n = count;
        if (count) AMGH_CUDA(cudaMalloc(&p, count * sizeof(T)));
    }
    void upload(const T* h, size_t count, cudaStream_t s) {
        alloc(count);
        if (count) AMGH_CUDA(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void upload(const std::vector<T>& v, cudaStream_t s) { upload(v.data(), v.size(), s); }
    void zero(cudaStream_t s) {
        if (n) AMGH_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
};

// CSR on the device (FP64 values)
struct DevCSR {
    int nrows = 0, ncols = 0;
    int64_t nnz = 0;
    int max_row = -1;   // longest row, when known (-1: unknown)
    DevArray<int32_t> ptr, idx;
    DevArray<double> val;
};

// Sliced ELL with slices of 32 consecutive rows, column-major inside a slice:
// entry t of row 32 s + lane lives at slice_ptr[s] + 32 t + lane; padding has value 0.
template <class V>
struct Sell {
    int nrows = 0, nslices = 0;
    int64_t stored = 0;                 // entries incl. padding
    DevArray<int64_t> slice_ptr;        // nslices + 1
    DevArray<int32_t> col;
    DevArray<V> val;
};

template <class V>
struct SellView {
    int nrows, nslices;
    const int64_t* __restrict__ slice_ptr;
    const int32_t* __restrict__ col;
    const V* __restrict__ val;
};

template <class V>
inline SellView<V> view(const Sell<V>& s) {
    return {s.nrows, s.nslices, s.slice_ptr.p, s.col.p, s.val.p};
}

struct LevelHost {
    HostCSR A;            // values on host (needed by the next coarsening's strength test)
    HostCSR G;
    Coarsening cz;        // empty on the coarsest level
    StarLayout stars;
    HostCSR Pn;           // nodal interpolation of the commuting correction (interp CONSTRAINED)
};

}  // namespace amgh
