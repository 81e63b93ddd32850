// V-cycle engine, templated on the hierarchy's storage type V and vector/accumulation type T.
#pragma once
#include <functional>
#include <memory>

#include "kernels.h"

namespace amgh {

// kernel classes for the roofline timing
enum KernelKind { K_SCHWARZ = 0, K_L1 = 1, K_RESID = 2, K_RESTRICT = 3, K_PROLONG = 4, K_COARSE = 5, K_SPMV = 6, K_RR = 7 };

struct Profiler {
    bool enabled = false;
    int kind = 0, level = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
    size_t used = 0;                  // pairs recorded since the last harvest
    std::vector<double> bytes_used;   // bytes of each recorded pair
    int64_t launches = 0;
    double total_ms = 0.0, bytes = 0.0;
    bool capturing = false;
    int gen = 0;                      // bumped whenever the profiled kernel class changes
    ~Profiler() { clear(); }
    void clear() {
        for (auto& p : pool) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
        pool.clear();
        used = 0;
        bytes_used.clear();
    }
    bool match(int k, int l) const { return enabled && k == kind && l == level; }
    std::pair<cudaEvent_t, cudaEvent_t> next() {
        if (used == pool.size()) {
            cudaEvent_t a, b;
            AMGH_CUDA(cudaEventCreate(&a));
            AMGH_CUDA(cudaEventCreate(&b));
            pool.push_back({a, b});
        }
        return pool[used++];
    }
    void record(cudaEvent_t e, cudaStream_t s) {
        if (capturing) AMGH_CUDA(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
        else AMGH_CUDA(cudaEventRecord(e, s));
    }
    // accumulate the recorded pairs (the stream must have passed them)
    void harvest(size_t npairs) {
        for (size_t i = 0; i < npairs && i < pool.size(); ++i) {
            float ms = 0.f;
            AMGH_CUDA(cudaEventSynchronize(pool[i].second));
            AMGH_CUDA(cudaEventElapsedTime(&ms, pool[i].first, pool[i].second));
            total_ms += ms;
            bytes += bytes_used[i];
            launches++;
        }
    }
};

class EngineBase {
   public:
    virtual ~EngineBase() = default;
    // FP64 device buffers the V-cycle reads its input from and writes its output to
    virtual double* in64() = 0;
    virtual double* out64() = 0;
    // out64 = B in64, enqueued on s (asynchronous); returns the number of kernels launched
    virtual int64_t vcycle(cudaStream_t s) = 0;
    // enqueue the V-cycle's kernels on s (used while capturing a larger graph); returns launches
    virtual int64_t enqueue(cudaStream_t s) = 0;
    // single V-cycle steps on level l (test entry), FP64 device pointers
    virtual void level_apply(int l, int op, const double* f, const double* x, double* y, cudaStream_t s) = 0;
    virtual void capture(cudaStream_t s) = 0;
    virtual void release_graph() = 0;
    // zero the words of every grid barrier (after a barrier wait gave up)
    virtual void reset_barriers(cudaStream_t s) = 0;
    Profiler* prof = nullptr;
    size_t prof_pairs = 0;   // event pairs one V-cycle records
};

}  // namespace amgh
