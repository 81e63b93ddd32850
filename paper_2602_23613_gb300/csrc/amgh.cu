// libamgh: setup driver, V-cycle engine, Krylov solvers and the C-ABI entry points.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <type_traits>

#ifdef _OPENMP
#include <omp.h>
#endif

#include <cstdlib>
#include <map>
#include <tuple>
#include <mutex>
#include <condition_variable>
#include <thread>
#include <variant>

#include "engine.cuh"
#include "krylov_scratch.h"
#include "mlp.cuh"
#include "multi.cuh"
#include "splitmix.cuh"
#include "vcycle_kernels.h"

namespace amgh {

std::atomic<int64_t>& launch_counter() {
    static std::atomic<int64_t> c{0};
    return c;
}

struct StatusError {
    amgh_status st;
    std::string msg;
};

static double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static void upload_csr(const HostCSR& h, DevCSR& d, cudaStream_t s, bool values) {
    d.nrows = h.nrows;
    d.ncols = h.ncols;
    d.nnz = h.nnz();
    d.max_row = 0;
    for (int r = 0; r < h.nrows; ++r) d.max_row = std::max(d.max_row, h.ptr[r + 1] - h.ptr[r]);
    d.ptr.upload(h.ptr, s);
    d.idx.upload(h.idx, s);
    if (values) d.val.upload(h.val, s);
    else d.val.alloc(d.nnz);
}

// slice pointers of a 32-row SELL for the rows of a host pattern (or for listed rows)
static std::vector<int64_t> sell_slices(const HostCSR& M, const std::vector<int32_t>* rows) {
    const int64_t nrows = rows ? (int64_t)rows->size() : M.nrows;
    const int64_t ns = (nrows + 31) / 32;
    std::vector<int64_t> sp(ns + 1, 0);
    for (int64_t s = 0; s < ns; ++s) {
        int w = 0;
        for (int64_t q = 32 * s; q < std::min<int64_t>(nrows, 32 * s + 32); ++q) {
            int r = rows ? (*rows)[q] : (int)q;
            if (r >= 0) w = std::max(w, M.ptr[r + 1] - M.ptr[r]);
        }
        sp[s + 1] = sp[s] + 32 * (int64_t)w;
    }
    return sp;
}

template <class V>
static void build_sell(const HostCSR& pat, const DevCSR& dev, Sell<V>& S, cudaStream_t s) {
    auto sp = sell_slices(pat, nullptr);
    S.nrows = pat.nrows;
    S.nslices = (int)(sp.size() - 1);
    S.stored = sp.back();
    S.slice_ptr.upload(sp, s);
    S.col.alloc(S.stored);
    S.val.alloc(S.stored);
    launch_sell_fill<V>(dev, S, s);
}

// ---------------------------------------------------------------------------------------------
// V-cycle engine: every level carries its own storage precision (FP64, or FP32 / BF16 with FP32
// vectors) and its own layouts, chosen at setup by the precision policy and the autotuner.
// ---------------------------------------------------------------------------------------------
// V: storage of the level (star rows, block inverses, A, P, P^T and W = P^T A), decided by the
// condition guard; T: vectors and accumulation.  AT names the storage the residual, l1-Jacobi and
// transfer passes read (the same V).
template <class V, class T, class VA = V>
struct LevelX {
    using VT = V;
    using TT = T;
    using AT = VA;
    int n = 0;
    SellL<VA> A, P, PT, W;
    bool fuse_rr = false;     // residual + restriction as one pass over P^T and W
    SmootherL<V> sm;
    DevArray<T> l1inv, f, x, y, r;
    int64_t nnzA = 0, nnzP = 0, nnzW = 0;
    std::vector<int64_t> col_nnz, col_inv, col_rows;   // per colour, for the algorithmic bytes
};
using bf16 = __nv_bfloat16;
using LevelVar = std::variant<LevelX<double, double>, LevelX<float, float>, LevelX<bf16, float>>;

// whether a level's vectors are FP64
static bool vectors_double(const LevelVar& v) {
    return std::visit([](const auto& d) { return std::is_same<typename std::decay_t<decltype(d)>::TT, double>::value; },
                      v);
}

struct LevelChoice {
    int prec = AMGH_F64;
    int L_A = 1, L_P = 1, L_PT = 1, L_sm = 1;
    bool fused = false;
    int persist = 0;   // grid of the cooperative whole-sweep launch, 0: not used
    bool staged = false;   // that launch stages its chunks in shared memory
    bool cluster = false;  // ... and runs as one thread-block cluster (hardware barrier)
    int stream = 0;        // per-colour streaming launches of at most this many CTAs, 0: not used
    int stream_bufs = 2;   // their stage buffers per CTA
    bool pdl = false;      // per-colour launches with programmatic dependent launch
    int cluster2 = 0;      // register-prefetching sweep in one cluster of this many 512-thread CTAs
    int resident = 0;      // sweep with x in shared memory in one cluster of this many CTAs
    int resident_g = 1;    // ... of this many 256-thread chunk groups each
    bool resident_grid = false;   // ... as a cooperative grid of `resident` CTAs with x in global memory
    double kappa = 0.0;
    bool fuse_rr = false;    // residual + restriction fused into one pass over P^T and W = P^T A
    int L_RR = 1;            // lanes per row of that pass (P^T and W share it)
};

struct Engine : EngineBase {
    std::vector<LevelVar> L;
    std::vector<LevelChoice> choice;
    int nlev = 0, nL = 0;
    DevArray<double> cinv_d;
    DevArray<float> cinv_f;
    int tail = -1;                     // level whose whole sub-cycle is applied as a dense operator
    DevArray<double> tail_d;
    DevArray<float> tail_f;
    DevArray<double> io_in, io_out;   // FP64 staging when level 0 stores float vectors
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool prof_in_graph = false;
    int prof_gen = -1;
    int64_t launches_vc = 0;

    ~Engine() override { release_graph(); }
    void reset_barriers(cudaStream_t s) override {
        for (auto& v : L)
            std::visit([&](auto& d) {
                if (d.sm.bar.p) d.sm.bar.zero(s);
            }, v);
    }

    bool level0_double() const { return vectors_double(L[0]); }
    // level 0's buffers as FP64 (null when its vectors are float)
    template <class Pick>
    double* level0_buf(Pick pick) {
        return std::visit([&](auto& d) -> double* {
            if constexpr (std::is_same<typename std::decay_t<decltype(d)>::TT, double>::value) return pick(d);
            else return nullptr;
        }, L[0]);
    }
    double* in64() override {
        return level0_double() ? level0_buf([](auto& d) { return d.f.p; }) : io_in.p;
    }
    double* out64() override {
        return level0_double() ? level0_buf([](auto& d) { return d.x.p; }) : io_out.p;
    }

    template <class F>
    void timed(int kind, int level, double bytes, cudaStream_t s, F&& fn) {
        if (prof && prof->match(kind, level)) {
            auto ev = prof->next();
            prof->bytes_used.resize(prof->used);
            prof->bytes_used[prof->used - 1] = bytes;
            prof->record(ev.first, s);
            fn();
            prof->record(ev.second, s);
        } else {
            fn();
        }
    }

    static std::vector<int> colour_sequence(int nc) {
        std::vector<int> seq;
        for (int c = 0; c < nc; ++c) seq.push_back(c);
        for (int c = nc - 2; c >= 0; --c) seq.push_back(c);
        return seq;
    }

    template <class Lv>
    double bytes_pass(const Lv& d, int64_t nnz, int64_t rows, int vecs) const {
        using V = typename Lv::AT;
        using T = typename Lv::TT;
        return (double)nnz * (sizeof(V) + 4) + 4.0 * rows + (double)vecs * sizeof(T) * rows;
    }
    template <class Lv>
    double bytes_colour(const Lv& d, int c) const {
        using V = typename Lv::VT;
        using T = typename Lv::TT;
        return (double)d.col_nnz[c] * (sizeof(V) + 4) + (double)d.col_inv[c] * sizeof(V) +
               3.0 * sizeof(T) * d.col_rows[c];
    }

    template <class Lv>
    void sweep(Lv& d, int l, cudaStream_t s, int64_t& cnt) {
        using V = typename Lv::VT;
        using T = typename Lv::TT;
        if (d.sm.fused || d.sm.persist > 0) {
            double by = 0;
            for (int c : colour_sequence(d.sm.ncolours)) by += bytes_colour(d, c);
            timed(K_SCHWARZ, l, by, s, [&] {
                if (d.sm.fused) launch_schwarz_fused<V, T>(d.sm, d.f.p, d.x.p, s);
                else launch_schwarz_persistent<V, T>(d.sm, d.f.p, d.x.p, s);
            });
            cnt++;
            return;
        }
        for (int c : colour_sequence(d.sm.ncolours)) {
            timed(K_SCHWARZ, l, bytes_colour(d, c), s, [&] { launch_schwarz_colourL<V, T>(d.sm, c, d.f.p, d.x.p, s); });
            cnt++;
        }
    }
    template <class Lv>
    void smooth_pre(Lv& d, int l, cudaStream_t s, int64_t& cnt) {
        using V = typename Lv::AT;
        using T = typename Lv::TT;
        sweep(d, l, s, cnt);
        timed(K_L1, l, bytes_pass(d, d.nnzA, d.n, 4), s,
              [&] { launch_sellL<V, T, T>(SM_L1, d.A, d.x.p, d.f.p, d.l1inv.p, d.y.p, s); });
        cnt++;
    }
    template <class Lv>
    void smooth_post(Lv& d, int l, cudaStream_t s, int64_t& cnt) {
        using V = typename Lv::AT;
        using T = typename Lv::TT;
        timed(K_L1, l, bytes_pass(d, d.nnzA, d.n, 4), s,
              [&] { launch_sellL<V, T, T>(SM_L1, d.A, d.y.p, d.f.p, d.l1inv.p, d.x.p, s); });
        cnt++;
        sweep(d, l, s, cnt);
    }

    // the fused pass's algorithmic bytes: P^T and W once each (values and columns, row pointers),
    // f and y of the fine level read once, the coarse right-hand side written once
    template <class Lv>
    double bytes_rr(const Lv& a, int64_t nc, size_t tb) const {
        using V = typename Lv::AT;
        using T = typename Lv::TT;
        return (double)(a.nnzP + a.nnzW) * (sizeof(V) + 4) + 8.0 * nc + 2.0 * sizeof(T) * a.n + (double)tb * nc;
    }

    int64_t core(cudaStream_t s) {
        int64_t cnt = 0;
        if (!level0_double()) {
            std::visit([&](auto& d) {
                using T = typename std::decay_t<decltype(d)>::TT;
                if constexpr (!std::is_same<T, double>::value) launch_convert<T>(io_in.p, d.f.p, (int64_t)d.n, s);
            }, L[0]);
            cnt++;
        }
        const int last = tail >= 0 ? tail : nlev - 1;
        for (int l = 0; l < last; ++l) {
            std::visit([&](auto& d) {
                using V = typename std::decay_t<decltype(d)>::AT;
                using T = typename std::decay_t<decltype(d)>::TT;
                d.x.zero(s);
                smooth_pre(d, l, s, cnt);
                if (d.fuse_rr) return;
                timed(K_RESID, l, bytes_pass(d, d.nnzA, d.n, 3), s,
                      [&] { launch_sellL<V, T, T>(SM_RESID, d.A, d.y.p, d.f.p, (const T*)nullptr, d.r.p, s); });
                cnt++;
            }, L[l]);
            std::visit([&](auto& a, auto& b) {
                using V = typename std::decay_t<decltype(a)>::AT;
                using Ta = typename std::decay_t<decltype(a)>::TT;
                using Tb = typename std::decay_t<decltype(b)>::TT;
                if (a.fuse_rr) {
                    timed(K_RR, l, bytes_rr(a, b.n, sizeof(Tb)), s,
                          [&] { launch_rr<V, Ta, Tb>(a.PT, a.W, a.f.p, a.y.p, b.f.p, s); });
                    cnt++;
                    return;
                }
                const double by = bytes_pass(a, a.nnzP, b.n, 0) + sizeof(Ta) * (double)a.n + sizeof(Tb) * (double)b.n;
                timed(K_RESTRICT, l, by, s, [&] {
                    launch_sellL<V, Ta, Tb>(SM_AX, a.PT, a.r.p, (const Tb*)nullptr, (const Tb*)nullptr, b.f.p, s);
                });
                cnt++;
            }, L[l], L[l + 1]);
        }
        std::visit([&](auto& d) {
            using T = typename std::decay_t<decltype(d)>::TT;
            const T* ci;
            if constexpr (std::is_same<T, double>::value) ci = last == nlev - 1 ? cinv_d.p : tail_d.p;
            else ci = last == nlev - 1 ? cinv_f.p : tail_f.p;
            const int m = d.n;
            timed(K_COARSE, last, (double)m * m * sizeof(T), s,
                  [&] { launch_coarse_apply<T>(ci, m, d.f.p, d.x.p, s); });
            cnt++;
        }, L[last]);
        for (int l = last - 1; l >= 0; --l) {
            std::visit([&](auto& a, auto& b) {
                using V = typename std::decay_t<decltype(a)>::AT;
                using Ta = typename std::decay_t<decltype(a)>::TT;
                using Tb = typename std::decay_t<decltype(b)>::TT;
                const double by = bytes_pass(a, a.nnzP, a.n, 2) + sizeof(Tb) * (double)b.n;
                timed(K_PROLONG, l, by, s, [&] {
                    launch_sellL<V, Tb, Ta>(SM_ADD, a.P, b.x.p, (const Ta*)nullptr, (const Ta*)nullptr, a.y.p, s);
                });
                cnt++;
            }, L[l], L[l + 1]);
            std::visit([&](auto& d) { smooth_post(d, l, s, cnt); }, L[l]);
        }
        if (!level0_double()) {
            std::visit([&](auto& d) {
                using T = typename std::decay_t<decltype(d)>::TT;
                if constexpr (!std::is_same<T, double>::value) launch_to_double<T>(d.x.p, io_out.p, (int64_t)d.n, s);
            }, L[0]);
            cnt++;
        }
        return cnt;
    }

    int64_t enqueue(cudaStream_t s) override { return core(s); }

    int64_t vcycle(cudaStream_t s) override {
        const bool want_prof = prof && prof->enabled;
        if (!gexec || want_prof != prof_in_graph || (want_prof && prof_gen != prof->gen)) capture(s);
        if (want_prof && prof_pairs) {
            // every replay records into fresh event pairs, so that a solve harvests them once at
            // its end instead of synchronising after every V-cycle
            const size_t base = prof->used;
            for (size_t i = 0; i < prof_pairs; ++i) prof->next();
            prof->bytes_used.resize(prof->used);
            for (size_t i = 0; i < prof_pairs; ++i) prof->bytes_used[base + i] = prof_bytes[i];
            for (const auto& pn : prof_nodes) {
                const auto& pr = prof->pool[base + pn.pair];
                AMGH_CUDA(cudaGraphExecEventRecordNodeSetEvent(gexec, pn.node, pn.second ? pr.second : pr.first));
            }
        }
        AMGH_CUDA(cudaGraphLaunch(gexec, s));
        launch_counter().fetch_add(launches_vc);
        return launches_vc;
    }

    struct ProfNode {
        cudaGraphNode_t node;
        size_t pair;
        bool second;
    };
    std::vector<ProfNode> prof_nodes;   // event-record nodes of the captured V-cycle, by pair
    std::vector<double> prof_bytes;     // algorithmic bytes of each pair

    void capture(cudaStream_t s) override {
        release_graph();
        prof_in_graph = prof && prof->enabled;
        prof_gen = prof ? prof->gen : -1;
        if (prof) { prof->used = 0; prof->capturing = true; }
        const int64_t before = launch_counter().load();   // capturing launches nothing
        AMGH_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int64_t cnt = 0;
        try {
            cnt = core(s);
        } catch (...) {
            cudaGraph_t g;
            cudaStreamEndCapture(s, &g);
            if (g) cudaGraphDestroy(g);
            if (prof) prof->capturing = false;
            launch_counter().store(before);
            throw;
        }
        AMGH_CUDA(cudaStreamEndCapture(s, &graph));
        launch_counter().store(before);
        prof_nodes.clear();
        prof_bytes.clear();
        if (prof) {
            prof->capturing = false;
            prof_pairs = prof->used;
            prof_bytes.assign(prof->bytes_used.begin(), prof->bytes_used.begin() + prof_pairs);
            if (prof_pairs) {
                size_t nn = 0;
                AMGH_CUDA(cudaGraphGetNodes(graph, nullptr, &nn));
                std::vector<cudaGraphNode_t> nodes(nn);
                AMGH_CUDA(cudaGraphGetNodes(graph, nodes.data(), &nn));
                for (cudaGraphNode_t nd : nodes) {
                    cudaGraphNodeType ty;
                    AMGH_CUDA(cudaGraphNodeGetType(nd, &ty));
                    if (ty != cudaGraphNodeTypeEventRecord) continue;
                    cudaEvent_t ev = nullptr;
                    AMGH_CUDA(cudaGraphEventRecordNodeGetEvent(nd, &ev));
                    for (size_t i = 0; i < prof_pairs; ++i) {
                        if (prof->pool[i].first == ev) prof_nodes.push_back({nd, i, false});
                        if (prof->pool[i].second == ev) prof_nodes.push_back({nd, i, true});
                    }
                }
            }
            prof->used = 0;
        }
        AMGH_CUDA(cudaGraphInstantiate(&gexec, graph, 0));
        launches_vc = cnt;
    }

    void release_graph() override {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
    }

    void level_apply(int l, int op, const double* f, const double* x, double* y, cudaStream_t s) override {
        if (op == 6) l = nlev - 1;
        if (l < 0 || l >= nlev || (op != 6 && l == nlev - 1))
            throw StatusError{AMGH_ERR_INVALID_ARG, "level out of range for this operation"};
        auto in = [&](const double* src, auto* dst, int64_t cnt) {
            using T = std::remove_pointer_t<decltype(dst)>;
            launch_convert<T>(src, dst, cnt, s);
        };
        auto out = [&](const auto* src, double* dst, int64_t cnt) {
            using T = std::remove_cv_t<std::remove_pointer_t<decltype(src)>>;
            launch_to_double<T>(src, dst, cnt, s);
        };
        if (op == 4 || op == 5 || op == 7) {
            std::visit([&](auto& a, auto& b) {
                using V = typename std::decay_t<decltype(a)>::AT;
                using Ta = typename std::decay_t<decltype(a)>::TT;
                using Tb = typename std::decay_t<decltype(b)>::TT;
                if (op == 7) {
                    if (a.W.nrows != a.PT.nrows || a.W.nslices != a.PT.nslices)
                        throw StatusError{AMGH_ERR_INVALID_ARG, "level " + std::to_string(l) +
                                                                    " holds no W = P^T A (fused restriction off)"};
                    in(f, a.f.p, a.n);
                    in(x, a.y.p, a.n);
                    launch_rr<V, Ta, Tb>(a.PT, a.W, a.f.p, a.y.p, b.f.p, s);
                    out(b.f.p, y, b.n);
                } else if (op == 4) {
                    in(x, a.r.p, a.n);
                    launch_sellL<V, Ta, Tb>(SM_AX, a.PT, a.r.p, (const Tb*)nullptr, (const Tb*)nullptr, b.f.p, s);
                    out(b.f.p, y, b.n);
                } else {
                    in(x, b.x.p, b.n);
                    in(y, a.y.p, a.n);
                    launch_sellL<V, Tb, Ta>(SM_ADD, a.P, b.x.p, (const Ta*)nullptr, (const Ta*)nullptr, a.y.p, s);
                    out(a.y.p, y, a.n);
                }
            }, L[l], L[l + 1]);
            return;
        }
        std::visit([&](auto& d) {
            using V = typename std::decay_t<decltype(d)>::AT;
            using T = typename std::decay_t<decltype(d)>::TT;
            int64_t c = 0;
            switch (op) {
                case 0:
                case 1:
                    in(x, d.x.p, d.n);
                    if (op == 1) in(f, d.f.p, d.n);
                    launch_sellL<V, T, T>(op == 0 ? SM_AX : SM_RESID, d.A, d.x.p, d.f.p, (const T*)nullptr, d.r.p, s);
                    out(d.r.p, y, d.n);
                    break;
                case 2:
                    in(x, d.x.p, d.n);
                    in(f, d.f.p, d.n);
                    smooth_pre(d, l, s, c);
                    out(d.y.p, y, d.n);
                    break;
                case 3:
                    in(x, d.y.p, d.n);
                    in(f, d.f.p, d.n);
                    smooth_post(d, l, s, c);
                    out(d.x.p, y, d.n);
                    break;
                case 6: {
                    const T* ci;
                    if constexpr (std::is_same<T, double>::value) ci = cinv_d.p;
                    else ci = cinv_f.p;
                    in(x, d.f.p, d.n);
                    launch_coarse_apply<T>(ci, nL, d.f.p, d.x.p, s);
                    out(d.x.p, y, d.n);
                    break;
                }
                default:
                    throw StatusError{AMGH_ERR_INVALID_ARG, "unknown level operation"};
            }
        }, L[l]);
    }
};

// ---------------------------------------------------------------------------------------------
// Multi-right-hand-side V-cycle (FP64, row-major K-wide vectors) on the hierarchy's FP64 CSR
// matrices: every level's Schwarz colours, l1-Jacobi, transfers and the coarsest inverse for K
// right-hand sides at once.
// ---------------------------------------------------------------------------------------------
struct MultiEngine {
    std::vector<MultiLevel> L;
    int nlev = 0, nL = 0, KP = 0;
    const double* cinv = nullptr;
    DevArray<double> partial, colv;     // per-column partial sums / results

    static std::vector<int> colour_sequence(int nc) {
        std::vector<int> seq;
        for (int c = 0; c < nc; ++c) seq.push_back(c);
        for (int c = nc - 2; c >= 0; --c) seq.push_back(c);
        return seq;
    }

    int first_built = 0;   // levels below it carry no smoother (built for a dense tail only)

    // smoother structures of levels >= first (a dense tail needs only its own sub-cycle).  prec:
    // storage of each level (AMGH_F64, or reduced: FP32 values and vectors); null = all FP64
    void build(const std::vector<LevelHost>& hl, const std::vector<DevCSR>& A64, const std::vector<DevCSR>& P64,
               const std::vector<DevCSR>& PT64, const double* cinv64, int* err, cudaStream_t s, int first = 0,
               const std::vector<int>* prec = nullptr) {
        nlev = (int)hl.size();
        first_built = first;
        width.clear();
        L.clear();
        L.resize(nlev);
        for (int l = 0; l < nlev; ++l) {
            MultiLevel& d = L[l];
            d.n = hl[l].A.nrows;
            d.A = &A64[l];
            d.f32 = prec && l < (int)prec->size() && (*prec)[l] != AMGH_F64;
            if (l + 1 == nlev) break;
            d.P = &P64[l];
            d.PT = &PT64[l];
            if (l < first) continue;
            const StarLayout& st = hl[l].stars;
            d.ncolours = st.ncolours;
            d.bmax = std::max(1, st.max_block);
            std::vector<int32_t> list;
            d.colour_star_begin.assign(st.ncolours + 1, 0);
            for (int c = 0; c < st.ncolours; ++c) {
                d.colour_star_begin[c] = (int32_t)list.size();
                for (int j = 0; j < st.nstars; ++j)
                    if (st.colour[j] == c && st.star_ptr[j + 1] > st.star_ptr[j]) list.push_back(j);
            }
            d.colour_star_begin[st.ncolours] = (int32_t)list.size();
            d.star_list.upload(list, s);
            // long rows: colour steps in split-K form over the rows of the colour's stars
            d.splitk = hl[l].A.nrows > 0 && hl[l].A.nnz() >= 64 * (int64_t)hl[l].A.nrows;
            if (d.splitk) {
                std::vector<int32_t> crow, cstar, cq, cbase;
                d.colour_row_begin.assign(st.ncolours + 1, 0);
                d.max_colour_rows = 0;
                for (int c = 0; c < st.ncolours; ++c) {
                    d.colour_row_begin[c] = (int32_t)crow.size();
                    for (int u = d.colour_star_begin[c]; u < d.colour_star_begin[c + 1]; ++u) {
                        const int j = list[u];
                        const int base = (int)crow.size() - d.colour_row_begin[c];
                        for (int q = 0; q < st.star_ptr[j + 1] - st.star_ptr[j]; ++q) {
                            crow.push_back(st.star_idx[st.star_ptr[j] + q]);
                            cstar.push_back(j);
                            cq.push_back(q);
                            cbase.push_back(base);
                        }
                    }
                    d.max_colour_rows = std::max(d.max_colour_rows, (int)crow.size() - d.colour_row_begin[c]);
                }
                d.colour_row_begin[st.ncolours] = (int32_t)crow.size();
                d.crow.upload(crow, s);
                d.cstar.upload(cstar, s);
                d.cq.upload(cq, s);
                d.cbase.upload(cbase, s);
            }
            d.star_ptr.upload(st.star_ptr, s);
            d.star_idx.upload(st.star_idx, s);
            std::vector<int64_t> off(st.nstars + 1, 0);
            for (int j = 0; j < st.nstars; ++j) {
                const int64_t b = st.star_ptr[j + 1] - st.star_ptr[j];
                off[j + 1] = off[j] + b * b;
            }
            d.inv_off.upload(off, s);
            d.inv.alloc(std::max<int64_t>(1, off.back()));
            launch_star_inverse_rowmajor(A64[l], st.nstars, d.star_ptr.p, d.star_idx.p, d.inv_off.p, d.inv.p, err, s);
            d.l1inv.alloc(d.n);
            launch_l1inv<double>(A64[l], d.l1inv.p, s);
            if (d.f32) {   // FP32 copies of the level's values (rounded once from FP64)
                auto narrow = [&](const double* src, size_t cnt, DevArray<float>& dst) {
                    dst.alloc(std::max<size_t>(1, cnt));
                    if (cnt) launch_convert<float>(src, dst.p, (int64_t)cnt, s);
                };
                narrow(A64[l].val.p, (size_t)A64[l].nnz, d.Af);
                narrow(P64[l].val.p, (size_t)P64[l].nnz, d.Pf);
                narrow(PT64[l].val.p, (size_t)PT64[l].nnz, d.PTf);
                narrow(d.inv.p, (size_t)off.back(), d.invf);
                narrow(d.l1inv.p, (size_t)d.n, d.l1invf);
            }
        }
        nL = hl.back().A.nrows;
        cinv = cinv64;
        AMGH_CUDA(cudaStreamSynchronize(s));
    }

    bool any_f32() const {
        for (const MultiLevel& d : L)
            if (d.f32) return true;
        return false;
    }

    std::vector<int> width;   // allocated width of each level's vectors (0 = none)

    // vectors of levels >= first at width kp (levels above `first` are left alone)
    void ensure_width(int kp, int first = 0) {
        if ((int)width.size() != (int)L.size()) width.assign(L.size(), 0);
        KP = kp;
        for (size_t l = first; l < L.size(); ++l) {
            if (width[l] == kp) continue;
            MultiLevel& d = L[l];
            const size_t nk = (size_t)d.n * kp, rk = (size_t)std::max(1, d.max_colour_rows) * kp;
            if (d.f32) {
                d.Ff.alloc(nk);
                d.Xf.alloc(nk);
                d.Yf.alloc(nk);
                d.Rf.alloc(nk);
                if (d.splitk) d.Rcf.alloc(rk);
            } else {
                d.F.alloc(nk);
                d.X.alloc(nk);
                d.Y.alloc(nk);
                d.R.alloc(nk);
                if (d.splitk) d.Rc.alloc(rk);
            }
            width[l] = kp;
        }
        if (partial.n != (size_t)304 * kp) {
            partial.alloc((size_t)304 * kp);
            colv.alloc(kp);
        }
    }

    // one level's arrays in its storage type
    template <class T>
    struct View {
        using type = T;
        const T *A, *P, *PT, *inv, *l1inv;
        T *F, *X, *Y, *R, *Rc;
    };
    static View<double> view64(MultiLevel& d) {
        return {d.A ? d.A->val.p : nullptr, d.P ? d.P->val.p : nullptr, d.PT ? d.PT->val.p : nullptr, d.inv.p,
                d.l1inv.p, d.F.p, d.X.p, d.Y.p, d.R.p, d.Rc.p};
    }
    static View<float> view32(MultiLevel& d) {
        return {d.Af.p, d.Pf.p, d.PTf.p, d.invf.p, d.l1invf.p, d.Ff.p, d.Xf.p, d.Yf.p, d.Rf.p, d.Rcf.p};
    }
    template <class Fn>
    static void typed(MultiLevel& d, Fn&& fn) {
        if (d.f32) fn(view32(d));
        else fn(view64(d));
    }

    // X_t = (V-cycle restricted to levels t..) F_t, for the KP columns of level t's F; every level
    // works in its own storage type, transfers between levels convert on the fly
    int64_t vcycle_from(int t, cudaStream_t s) {
        int64_t cnt = 0;
        for (int l = t; l + 1 < nlev; ++l) {
            MultiLevel& d = L[l];
            typed(d, [&](auto v) {
                using T = typename decltype(v)::type;
                AMGH_CUDA(cudaMemsetAsync(v.X, 0, sizeof(T) * d.n * KP, s));
                for (int c : colour_sequence(d.ncolours)) {
                    launch_schwarz_multi_t<T>(d, v.A, v.inv, v.Rc, c, KP, v.F, v.X, s);
                    cnt++;
                }
                launch_spmm_t<T, T, T>(MM_L1, d.n, d.A->ptr.p, d.A->idx.p, v.A, KP, v.X, v.F, v.l1inv, v.Y, s);
                launch_spmm_t<T, T, T>(MM_RESID, d.n, d.A->ptr.p, d.A->idx.p, v.A, KP, v.Y, v.F, (const T*)nullptr,
                                       v.R, s);
                typed(L[l + 1], [&](auto w) {
                    using U = typename decltype(w)::type;
                    launch_spmm_t<T, T, U>(MM_AX, d.PT->nrows, d.PT->ptr.p, d.PT->idx.p, v.PT, KP, v.R,
                                           (const U*)nullptr, (const U*)nullptr, w.F, s);
                });
                cnt += 3;
            });
        }
        typed(L[nlev - 1], [&](auto w) {
            using U = typename decltype(w)::type;
            launch_dense_apply_multi_t<U, U>(cinv, nL, KP, w.F, w.X, s);
        });
        cnt++;
        for (int l = nlev - 2; l >= t; --l) {
            MultiLevel& d = L[l];
            typed(d, [&](auto v) {
                using T = typename decltype(v)::type;
                typed(L[l + 1], [&](auto w) {
                    using U = typename decltype(w)::type;
                    launch_spmm_t<T, U, T>(MM_ADD, d.P->nrows, d.P->ptr.p, d.P->idx.p, v.P, KP, w.X, (const T*)nullptr,
                                           (const T*)nullptr, v.Y, s);
                });
                launch_spmm_t<T, T, T>(MM_L1, d.n, d.A->ptr.p, d.A->idx.p, v.A, KP, v.Y, v.F, v.l1inv, v.X, s);
                cnt += 2;
                for (int c : colour_sequence(d.ncolours)) {
                    launch_schwarz_multi_t<T>(d, v.A, v.inv, v.Rc, c, KP, v.F, v.X, s);
                    cnt++;
                }
            });
        }
        return cnt;
    }

    // level 0's right-hand side from a row-major FP64 block (n x KP), and its result back
    void load_rhs(const double* R, cudaStream_t s) {
        MultiLevel& d = L[0];
        if (d.f32) launch_convert<float>(R, d.Ff.p, (int64_t)d.n * KP, s);
        else if (R != d.F.p) AMGH_CUDA(cudaMemcpyAsync(d.F.p, R, sizeof(double) * d.n * KP, cudaMemcpyDeviceToDevice, s));
    }
    void store_result(double* Z, cudaStream_t s) {
        MultiLevel& d = L[0];
        if (d.f32) launch_widen(d.Xf.p, (int64_t)d.n * KP, Z, s);
        else if (Z != d.X.p) AMGH_CUDA(cudaMemcpyAsync(Z, d.X.p, sizeof(double) * d.n * KP, cudaMemcpyDeviceToDevice, s));
    }

    // dense operator of the V-cycle restricted to levels t.. (row-major n_t x n_t), column blocks
    void dense_tail(int t, DevArray<double>& B, cudaStream_t s) {
        const int nt = L[t].n;
        B.alloc((size_t)nt * nt);
        // a multiple of 256 columns: eight per lane in the multi-RHS kernels
        const int kp = std::min(2048, ((nt + 255) / 256) * 256);
        ensure_width(kp, t);
        std::vector<double> eye((size_t)nt * kp);
        for (int c0 = 0; c0 < nt; c0 += kp) {
            const int cnt = std::min(kp, nt - c0);
            std::fill(eye.begin(), eye.end(), 0.0);
            for (int c = 0; c < cnt; ++c) eye[(size_t)(c0 + c) * kp + c] = 1.0;
            AMGH_CUDA(cudaMemcpyAsync(L[t].F.p, eye.data(), sizeof(double) * eye.size(), cudaMemcpyHostToDevice, s));
            vcycle_from(t, s);
            AMGH_CUDA(cudaMemcpy2DAsync(B.p + c0, sizeof(double) * nt, L[t].X.p, sizeof(double) * kp,
                                        sizeof(double) * cnt, nt, cudaMemcpyDeviceToDevice, s));
            AMGH_CUDA(cudaStreamSynchronize(s));
        }
    }
};

}  // namespace amgh

using namespace amgh;

struct amgh_ctx {
    amgh_params prm{};
    cudaStream_t s = nullptr;
    std::string err;
    std::vector<LevelHost> hl;
    std::vector<DevCSR> A64, P64, PT64;
    std::vector<DevCSR> W64;              // W_l = P_l^T A_l for the fused residual + restriction
    std::vector<HostCSR> Wrows;           // its row pointers on the host (the SELL-L slice widths)
    DevArray<double> cinv64;
    std::unique_ptr<EngineBase> eng;
    std::unique_ptr<MultiEngine> meng;   // built on the first multi-RHS call (or for a dense tail)
    DevArray<double> dense_tail_B;       // dense operator of the V-cycle below the tail level
    int dense_tail_level = -1;
    Sell<double> A0;   // outer FP64 SpMV
    int64_t nnzA0 = 0;
    DevArray<double> kp, kq, kro, partial, scal, stage_f, stage_x;
    DevArray<int> iter;
    // device-resident solve graph (rebuilt when its pointers or parameters change)
    cudaGraph_t sgraph = nullptr;
    cudaGraphExec_t sexec = nullptr;
    const double* s_f = nullptr;
    double* s_x = nullptr;
    double s_tol = -1.0;
    int s_maxit = -1;
    int64_t s_pro_launches = 0, s_body_launches = 0;
    void drop_solve_graph() {
        if (sexec) cudaGraphExecDestroy(sexec);
        if (sgraph) cudaGraphDestroy(sgraph);
        sexec = nullptr;
        sgraph = nullptr;
        s_f = nullptr;
        s_x = nullptr;
    }
    double* hscal = nullptr;
    DevArray<int> errflag;
    DevArray<int> waitflag;          // raised by a device-side barrier wait that gave up
    DevArray<int> symflag;           // overflow flag of the symbolic product
    int nsm = 0;
    int dev = -1;                     // device current at setup; the handle's memory lives there
    Profiler prof;
    int64_t launches = 0;
    double host_ms = 0, dev_ms = 0;
    bool vc_pending = false;          // a V-cycle ran since the last harvest of its event pairs
    std::vector<int> max_patch;
    bool own_stream = false;
    bool structure_only = false;
    int interp_used = AMGH_INTERP_LOCAL;
    double rho_used = 0.0, rho_exact = 0.0, interp_ms = 0.0;
    bool host_loop = false;   // force the host-driven Krylov loop
    ~amgh_ctx() {
        drop_solve_graph();
        eng.reset();
        meng.reset();
        if (hscal) cudaFreeHost(hscal);
        if (own_stream && s) cudaStreamDestroy(s);
    }
};

struct amgh_mlp_ctx {
    MlpNet net;
    cudaStream_t s = nullptr;
    std::string err;
    ~amgh_mlp_ctx() {
        if (s) cudaStreamDestroy(s);
    }
};

static thread_local std::string g_setup_error;

namespace amgh {

// ---------------------------------------------------------------------------------------------
// Engine construction: precision policy, layouts and the autotuner
// ---------------------------------------------------------------------------------------------

// Pack the stars of every colour, without splitting a star, into chunks of 256/L row slots.
static StarPacking pack_stars(const StarLayout& st, int L) {
    StarPacking pk;
    pk.L = L;
    pk.slots = CTA_THREADS / L;
    pk.colour_cta_begin.assign(st.ncolours + 1, 0);
    pk.star_cta.assign(st.nstars, 0);
    pk.star_base.assign(st.nstars, 0);
    int nctas = 0;
    for (int c = 0; c < st.ncolours; ++c) {
        pk.colour_cta_begin[c] = nctas;
        int used = pk.slots;   // forces a new chunk for the colour's first star
        for (int j = 0; j < st.nstars; ++j) {
            if (st.colour[j] != c) continue;
            const int b = st.star_ptr[j + 1] - st.star_ptr[j];
            if (b == 0) continue;
            if (used + b > pk.slots) {
                nctas++;
                const size_t base = (size_t)(nctas - 1) * pk.slots;
                pk.slot_row.resize(base + pk.slots, -1);
                pk.slot_star.resize(base + pk.slots, -1);
                pk.slot_base.resize(base + pk.slots, 0);
                pk.slot_bsize.resize(base + pk.slots, 0);
                used = 0;
            }
            const size_t base = (size_t)(nctas - 1) * pk.slots;
            for (int q = 0; q < b; ++q) {
                pk.slot_row[base + used + q] = st.star_idx[st.star_ptr[j] + q];
                pk.slot_star[base + used + q] = j;
                pk.slot_base[base + used + q] = (int16_t)used;
                pk.slot_bsize[base + used + q] = (int8_t)b;
            }
            pk.star_cta[j] = nctas - 1;
            pk.star_base[j] = used;
            used += b;
        }
    }
    pk.colour_cta_begin[st.ncolours] = nctas;
    pk.nctas = nctas;
    return pk;
}

// slice pointers of a SELL-L layout: rows[q] for q < count (or 0..nrows-1 when rows is null)
static std::vector<int64_t> sellL_slices(const HostCSR& M, const std::vector<int32_t>* rows, int L) {
    const int64_t count = rows ? (int64_t)rows->size() : M.nrows;
    const int R = 32 / L;
    const int64_t ns = (count + R - 1) / R;
    std::vector<int64_t> sp(ns + 1, 0);
    for (int64_t s = 0; s < ns; ++s) {
        int w = 0;
        for (int64_t q = R * s; q < std::min<int64_t>(count, R * s + R); ++q) {
            const int r = rows ? (*rows)[q] : (int)q;
            if (r >= 0) w = std::max(w, (M.ptr[r + 1] - M.ptr[r] + L - 1) / L);
        }
        sp[s + 1] = sp[s] + 32 * (int64_t)w;
    }
    return sp;
}

template <class V>
static void build_sellL(const HostCSR& pat, const DevCSR& dev, int L, SellL<V>& S, cudaStream_t s) {
    auto sp = sellL_slices(pat, nullptr, L);
    S.L = L;
    S.nrows = pat.nrows;
    S.nslices = (int)(sp.size() - 1);
    S.stored = sp.back();
    S.slice_ptr.upload(sp, s);
    S.col.alloc(S.stored);
    S.val.alloc(S.stored);
    launch_sellL_fill<V>(dev, S, s);
}

// the same for a matrix whose pattern lives on the device only (W = P^T A): the host holds its row
// pointers, which the slice widths need
template <class V>
static void build_sellL_rows(const HostCSR& rows, const DevCSR& dev, int L, SellL<V>& S, cudaStream_t s) {
    build_sellL<V>(rows, dev, L, S, s);
}

// name of a smoother launch mode (AMGH_SMOOTHER_MODE restricts the autotuner to one of them)
static std::string smoother_mode_name(const LevelChoice& m) {
    if (m.fused) return "fused";
    if (m.resident > 0) return m.resident_grid ? "pipeline" : "resident";
    if (m.cluster2 > 0) return "cluster2";
    if (m.persist > 0) return m.cluster ? "cluster" : m.staged ? "staged" : "persistent";
    if (m.stream > 0) return m.stream_bufs == 1 ? "stream1" : "stream2";
    return m.pdl ? "pdl" : "colour";
}

// the same with the shape of a resident or pipelined sweep: <name>-<CTAs>x<chunk groups>-L<lanes>
static std::string smoother_mode_detail(const LevelChoice& m) {
    if (m.fused || m.resident <= 0) return smoother_mode_name(m);
    return smoother_mode_name(m) + "-" + std::to_string(m.resident) + "x" + std::to_string(m.resident_g) + "-L" +
           std::to_string(m.L_sm);
}

// launch mode of a built smoother (the layout is the same for every mode)
template <class V>
static void set_smoother_mode(SmootherL<V>& sm, const LevelChoice& m) {
    sm.fused = m.fused;
    sm.resident = m.fused ? 0 : m.resident;
    sm.resident_g = m.resident_g;
    sm.resident_grid = m.resident_grid;
    sm.cluster2 = (m.fused || sm.resident > 0) ? 0 : m.cluster2;
    sm.persist = m.fused ? 0 : sm.resident > 0 ? sm.resident : sm.cluster2 > 0 ? sm.cluster2 : m.persist;
    sm.staged = sm.persist > 0 && sm.cluster2 == 0 && sm.resident == 0 && m.staged;
    sm.cluster = sm.staged && m.cluster;
    sm.stream_grid = (m.fused || sm.persist > 0) ? 0 : m.stream;
    sm.stream_bufs = m.stream_bufs;
    sm.pdl = !m.fused && sm.persist == 0 && sm.stream_grid == 0 && m.pdl;
}

template <class V>
static void build_smoother(amgh_ctx* h, int l, int L, bool fused, int persist, bool staged, SmootherL<V>& sm,
                           std::vector<int64_t>* cn, std::vector<int64_t>* ci, std::vector<int64_t>* cr,
                           cudaStream_t s) {
    const LevelHost& hl = h->hl[l];
    const StarLayout& st = hl.stars;
    StarPacking pk = pack_stars(st, L);
    sm.L = L;
    sm.slots = pk.slots;
    sm.nctas = pk.nctas;
    sm.bmax = std::max(1, st.max_block);
    sm.ncolours = st.ncolours;
    sm.n = (int)hl.A.nrows;
    sm.fused = fused;
    sm.persist = fused ? 0 : persist;
    sm.bar.alloc(4);
    sm.bar.zero(s);
    sm.wait_err = h->waitflag.p;
    sm.colour_cta_begin = pk.colour_cta_begin;
    sm.colour_cta_begin_d.upload(pk.colour_cta_begin, s);
    std::vector<int32_t> seq;
    for (int c = 0; c < st.ncolours; ++c) seq.push_back(c);
    for (int c = st.ncolours - 2; c >= 0; --c) seq.push_back(c);
    sm.sweep_d.upload(seq, s);
    sm.slot_row.upload(pk.slot_row, s);
    sm.slot_base.upload(pk.slot_base, s);
    sm.slot_bsize.upload(pk.slot_bsize, s);
    // slot rows as SELL-L slices, 8 per chunk
    std::vector<int32_t> rows_for_slices;   // row of each (slice-row) position
    auto sp = sellL_slices(hl.A, &pk.slot_row, L);
    sm.rows.L = L;
    sm.rows.nrows = (int)pk.slot_row.size();
    sm.rows.nslices = (int)(sp.size() - 1);
    sm.rows.stored = sp.back();
    sm.rows.slice_ptr.upload(sp, s);
    sm.wmax = 0;
    for (size_t q = 0; q + 1 < sp.size(); ++q) sm.wmax = std::max<int>(sm.wmax, (int)((sp[q + 1] - sp[q]) / 32));
    sm.staged = staged && sm.persist > 0;
    sm.rows.col.alloc(sm.rows.stored);
    sm.rows.val.alloc(sm.rows.stored);
    launch_slotL_fill<V>(h->A64[l], sm, s);
    sm.inv.alloc((size_t)sm.nctas * sm.bmax * sm.slots);
    sm.inv.zero(s);
    DevArray<int32_t> dsp, dsi, dsc, dsb;
    dsp.upload(st.star_ptr, s);
    dsi.upload(st.star_idx, s);
    dsc.upload(pk.star_cta, s);
    dsb.upload(pk.star_base, s);
    launch_star_inverseL<V>(h->A64[l], st.nstars, dsp.p, dsi.p, dsc.p, dsb.p, sm, h->errflag.p, s);
    AMGH_CUDA(cudaStreamSynchronize(s));
    sm.stored_rows_nnz = 0;
    if (cn) {
        cn->assign(st.ncolours, 0);
        ci->assign(st.ncolours, 0);
        cr->assign(st.ncolours, 0);
        for (int c = 0; c < st.ncolours; ++c)
            for (int k = pk.colour_cta_begin[c]; k < pk.colour_cta_begin[c + 1]; ++k)
                for (int q = 0; q < pk.slots; ++q) {
                    const int r = pk.slot_row[(size_t)k * pk.slots + q];
                    if (r < 0) continue;
                    (*cn)[c] += hl.A.ptr[r + 1] - hl.A.ptr[r];
                    (*ci)[c] += pk.slot_bsize[(size_t)k * pk.slots + q];
                    (*cr)[c] += 1;
                }
    }
}

// wall time of setup phases on stderr when AMGH_VERBOSE=1 (the stream is synchronised only then)
struct DevPhases {
    bool on = std::getenv("AMGH_VERBOSE") != nullptr;
    double t = now_ms();
    void mark(cudaStream_t s, const char* what, int l = -1) {
        if (!on) return;
        cudaStreamSynchronize(s);
        const double now = now_ms();
        if (l >= 0) std::fprintf(stderr, "[amgh] L%d %-25s %8.1f ms\n", l, what, now - t);
        else std::fprintf(stderr, "[amgh] %-28s %8.1f ms\n", what, now - t);
        t = now;
    }
};

// time fn() (enqueued on s): best of `reps` after one warm-up, in ms
template <class F>
static float time_best(cudaStream_t s, int reps, F&& fn) {
    cudaEvent_t a, b;
    AMGH_CUDA(cudaEventCreate(&a));
    AMGH_CUDA(cudaEventCreate(&b));
    fn();
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        AMGH_CUDA(cudaEventRecord(a, s));
        fn();
        AMGH_CUDA(cudaEventRecord(b, s));
        AMGH_CUDA(cudaEventSynchronize(b));
        float ms = 0.f;
        AMGH_CUDA(cudaEventElapsedTime(&ms, a, b));
        best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

// cooperative whole-sweep launches need the device's support, inside captured graphs too
static bool cooperative_ok(amgh_ctx* h) {
    static std::mutex mu;
    static std::map<int, bool> known;
    int dev = 0;
    AMGH_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto it = known.find(dev);
    if (it == known.end()) it = known.emplace(dev, cooperative_capture_works()).first;
    (void)h;
    return it->second;
}

// read and clear the flag a device-side barrier wait raises when it gives up
static bool take_wait_flag(amgh_ctx* h, cudaStream_t s) {
    int flag = 0;
    AMGH_CUDA(cudaMemcpyAsync(&flag, h->waitflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGH_CUDA(cudaStreamSynchronize(s));
    if (flag) h->waitflag.zero(s);
    return flag != 0;
}
static bool take_wait_flag(amgh_ctx* h) { return take_wait_flag(h, h->s); }

// after a solve: a barrier wait that gave up invalidates the result; reset the barriers and report
static void check_wait(amgh_ctx* h) {
    if (!take_wait_flag(h)) return;
    if (h->eng) h->eng->reset_barriers(h->s);
    AMGH_CUDA(cudaStreamSynchronize(h->s));
    throw StatusError{AMGH_ERR_TIMEOUT, "a grid barrier of the Schwarz sweep gave up waiting; the result is invalid"};
}

// time fn() as it runs in the V-cycle: captured once into a graph, best of `reps` replays after
// one warm-up replay, in ms
template <class F>
static float time_best_graph(cudaStream_t s, int reps, F&& fn) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    AMGH_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    fn();
    AMGH_CUDA(cudaStreamEndCapture(s, &g));
    const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    if (ie != cudaSuccess) {
        cudaGraphDestroy(g);
        throw CudaError{ie, "instantiating a tuning graph"};
    }
    const float ms = time_best(s, reps, [&] { AMGH_CUDA(cudaGraphLaunch(ge, s)); });
    cudaGraphExecDestroy(ge);
    cudaGraphDestroy(g);
    return ms;
}

static bool tuning_enabled() {
    const char* e = std::getenv("AMGH_TUNE");
    return !(e && std::string(e) == "0");
}

// process-wide cache of tuned choices, keyed by the shape of a level
static std::mutex g_tune_mu;
static std::map<std::string, LevelChoice> g_tune_cache;

static std::string tune_key(const LevelHost& hl, size_t value_bytes, size_t matrix_bytes, int fuse) {
    const char* forced = std::getenv("AMGH_SMOOTHER_MODE");
    return std::string(forced ? forced : "") + "|" + std::to_string(value_bytes) + "|" + std::to_string(matrix_bytes) +
           "|" + std::to_string(fuse) + "|" + std::to_string(hl.A.nrows) +
           "|" + std::to_string(hl.A.nnz()) + "|" + std::to_string(hl.stars.ncolours) + "|" +
           std::to_string(hl.cz.P.nnz());
}

static std::vector<int> lane_candidates(double avg_len, int n, int need_slots_for) {
    std::vector<int> out;
    for (int L : {1, 2, 4, 8, 16, 32}) {
        if (need_slots_for > 0 && CTA_THREADS / L < need_slots_for) continue;
        if (L > 1 && L > avg_len / 2.0) continue;
        // large levels with short rows (the finest): the FP64 pipe decides, keep L small; large
        // levels with long rows (a first coarse level) need lanes to fill the GPU in each step
        if (n > 400000 && L > 2 && avg_len < 64.0) continue;
        out.push_back(L);
    }
    if (out.empty()) out.push_back(1);
    return out;
}

template <class V, class T, class VA>
static void build_level(amgh_ctx* h, int l, LevelX<V, T, VA>& d, LevelChoice& ch, cudaStream_t s) {
    const LevelHost& hl = h->hl[l];
    DevPhases ph;
    d.n = hl.A.nrows;
    d.nnzA = hl.A.nnz();
    d.nnzP = hl.cz.P.nnz();
    const bool haveW = l < (int)h->W64.size() && h->W64[l].nrows > 0;
    d.nnzW = haveW ? h->W64[l].nnz : 0;
    d.f.alloc(d.n);
    d.x.alloc(d.n);
    d.y.alloc(d.n);
    d.r.alloc(d.n);
    d.f.zero(s);
    d.x.zero(s);
    d.y.zero(s);
    d.r.zero(s);
    d.l1inv.alloc(d.n);
    launch_l1inv<T>(h->A64[l], d.l1inv.p, s);
    const double avg = d.n ? (double)d.nnzA / d.n : 1.0;
    const double avgPT = hl.cz.PT.nrows ? (double)hl.cz.PT.nnz() / hl.cz.PT.nrows : 1.0;
    const std::string key = tune_key(hl, sizeof(V), sizeof(VA), haveW ? h->prm.fuse_restrict : 0);
    bool cached = false;
    if (tuning_enabled()) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            const double kap = ch.kappa;
            const int prec = ch.prec;
            ch = it->second;
            ch.kappa = kap;
            ch.prec = prec;
            cached = true;
        }
    }
    const bool tune = tuning_enabled() && !cached;
    // coarse-level vectors for P / P^T timing use this level's type on both sides
    DevArray<T> cvec;
    if (tune) {
        cvec.alloc(std::max(1, hl.cz.P.ncols));
        cvec.zero(s);
    }
    // ---- A (l1-Jacobi, residual) ----
    float best_resid = 1e30f, best_restrict = 1e30f;
    if (tune) {
        for (int Lc : lane_candidates(avg, d.n, 0)) {
            SellL<VA> cand;
            build_sellL<VA>(hl.A, h->A64[l], Lc, cand, s);
            const float ms = time_best(s, 3, [&] {
                launch_sellL<VA, T, T>(SM_RESID, cand, d.x.p, d.f.p, (const T*)nullptr, d.r.p, s);
            });
            if (ms < best_resid) { best_resid = ms; ch.L_A = Lc; }
        }
    }
    build_sellL<VA>(hl.A, h->A64[l], ch.L_A, d.A, s);
    ph.mark(s, "  A layout", l);
    // ---- P (prolongation) and P^T (restriction) ----
    if (tune) {
        float best = 1e30f;
        for (int Lc : {1, 2}) {
            SellL<VA> cand;
            build_sellL<VA>(hl.cz.P, h->P64[l], Lc, cand, s);
            const float ms = time_best(s, 3, [&] {
                launch_sellL<VA, T, T>(SM_ADD, cand, cvec.p, (const T*)nullptr, (const T*)nullptr, d.y.p, s);
            });
            if (ms < best) { best = ms; ch.L_P = Lc; }
        }
        for (int Lc : lane_candidates(avgPT, hl.cz.PT.nrows, 0)) {
            if (Lc > 8) continue;
            SellL<VA> cand;
            build_sellL<VA>(hl.cz.PT, h->PT64[l], Lc, cand, s);
            const float ms = time_best(s, 3, [&] {
                launch_sellL<VA, T, T>(SM_AX, cand, d.r.p, (const T*)nullptr, (const T*)nullptr, cvec.p, s);
            });
            if (ms < best_restrict) { best_restrict = ms; ch.L_PT = Lc; }
        }
        // the fused pass over P^T and W = P^T A, against the residual pass plus the restriction
        ch.fuse_rr = false;
        if (haveW) {
            const double avgW = hl.cz.PT.nrows ? (double)(d.nnzW + hl.cz.PT.nnz()) / hl.cz.PT.nrows : 1.0;
            float best_rr = 1e30f;
            for (int Lc : lane_candidates(avgW, hl.cz.PT.nrows, 0)) {
                SellL<VA> cpt, cw;
                build_sellL<VA>(hl.cz.PT, h->PT64[l], Lc, cpt, s);
                build_sellL_rows<VA>(h->Wrows[l], h->W64[l], Lc, cw, s);
                const float ms = time_best(s, 3, [&] { launch_rr<VA, T, T>(cpt, cw, d.f.p, d.y.p, cvec.p, s); });
                if (ms < best_rr) { best_rr = ms; ch.L_RR = Lc; }
            }
            ch.fuse_rr = h->prm.fuse_restrict > 0 || best_rr < best_resid + best_restrict;
            if (ph.on)
                std::fprintf(stderr, "[amgh] L%d residual %.4f + restriction %.4f ms, fused (L %d) %.4f ms -> %s\n", l,
                             best_resid, best_restrict, ch.L_RR, best_rr, ch.fuse_rr ? "fused" : "apart");
        }
    }
    if (haveW && !tuning_enabled()) {
        ch.fuse_rr = h->prm.fuse_restrict > 0;
        ch.L_RR = ch.L_PT;
    }
    d.fuse_rr = haveW && ch.fuse_rr;
    build_sellL<VA>(hl.cz.P, h->P64[l], ch.L_P, d.P, s);
    build_sellL<VA>(hl.cz.PT, h->PT64[l], d.fuse_rr ? ch.L_RR : ch.L_PT, d.PT, s);
    // W is kept when the fused pass runs, or when it is forced on (then every level has it)
    if (haveW && (d.fuse_rr || h->prm.fuse_restrict > 0)) build_sellL_rows<VA>(h->Wrows[l], h->W64[l], d.PT.L, d.W, s);
    ph.mark(s, "  P, P^T, W layouts", l);
    // ---- smoother ----
    // Each lane count is built once; its launch modes only differ in how the same layout is
    // swept: per-colour launches, per-colour streaming launches (chunks staged in shared memory),
    // one single-CTA launch (small levels), one cooperative launch over several grid sizes, and
    // one cooperative launch with staged chunks (levels with many colours).  Every candidate is
    // timed as a captured graph, the way the V-cycle runs it.
    if (tune) {
        float best = 1e30f, best_colour = 1e30f;
        LevelChoice colour_choice = ch;
        const bool small = d.nnzA <= 3000000 && d.n <= 60000;
        for (int Lc : lane_candidates(avg, d.n, hl.stars.max_block)) {
            SmootherL<V> cand;
            build_smoother<V>(h, l, Lc, false, 0, false, cand, nullptr, nullptr, nullptr, s);
            int maxc = 1;
            for (int c = 0; c < cand.ncolours; ++c)
                maxc = std::max(maxc, cand.colour_cta_begin[c + 1] - cand.colour_cta_begin[c]);
            std::vector<LevelChoice> modes;
            // every launch-mode field starts cleared: the best choice so far must not leak into
            // another lane count's candidates
            LevelChoice m0 = ch;
            m0.L_sm = Lc;
            m0.fused = false;
            m0.persist = 0;
            m0.staged = false;
            m0.cluster = false;
            m0.cluster2 = 0;
            m0.resident = 0;
            m0.resident_g = 1;
            m0.resident_grid = false;
            m0.stream = 0;
            m0.stream_bufs = 2;
            m0.pdl = false;
            modes.push_back(m0);
            {
                LevelChoice m = m0;
                m.pdl = true;
                modes.push_back(m);
            }
            for (int nb : {2, 1}) {
                const int scap = schwarz_stream_cap<V, T>(cand, nb);
                for (int g : {scap, 2 * h->nsm, h->nsm}) {
                    LevelChoice m = m0;
                    m.stream = std::min(g, scap);
                    m.stream_bufs = nb;
                    if (m.stream > 0 && std::none_of(modes.begin(), modes.end(), [&](const LevelChoice& q) {
                            return q.stream == m.stream && q.stream_bufs == nb;
                        }))
                        modes.push_back(m);
                }
            }
            if (small) {
                LevelChoice m = m0;
                m.fused = true;
                modes.push_back(m);
            }
            if (cand.ncolours >= 4 && cooperative_ok(h)) {
                const int cap = schwarz_persistent_cap<V, T>(Lc);
                std::vector<int> grids;
                for (int g : {maxc, 4 * h->nsm, 2 * h->nsm, h->nsm, h->nsm / 2, h->nsm / 4}) {
                    g = std::min(g, std::min(cap, maxc));
                    if (g >= 1 && std::find(grids.begin(), grids.end(), g) == grids.end()) grids.push_back(g);
                }
                for (int g : grids) {
                    LevelChoice m = m0;
                    m.persist = g;
                    modes.push_back(m);
                }
                cand.persist = maxc;
                if (schwarz_staged_cap<V, T>(cand) >= maxc) {
                    LevelChoice m = m0;
                    m.persist = maxc;
                    m.staged = true;
                    modes.push_back(m);
                }
            }
            if (cand.ncolours >= 4 && maxc <= 16 && schwarz_cluster2_ok<V, T>(cand, (maxc + 1) / 2)) {
                LevelChoice m = m0;
                m.cluster2 = (maxc + 1) / 2;
                modes.push_back(m);
            }
            // x resident in the shared memory of one cluster: levels whose iterate fits in a CTA
            if (cand.ncolours >= 4) {
                for (int size : {16, 8})
                    for (int groups : {1, 2})
                        if (schwarz_resident_ok<V, T>(cand, size, groups)) {
                            LevelChoice m = m0;
                            m.resident = size;
                            m.resident_g = groups;
                            modes.push_back(m);
                        }
            }
            // the same item walk over a cooperative grid (x in global memory, counter barrier)
            if (cand.ncolours >= 4 && cooperative_ok(h)) {
                for (int groups : {1, 2}) {
                    const int cap = schwarz_pipeline_cap<V, T>(cand, groups);
                    std::vector<int> grids;
                    for (int gsz : {(maxc + groups - 1) / groups, h->nsm, h->nsm / 2, h->nsm / 4}) {
                        gsz = std::min(gsz, cap);
                        if (gsz >= 1 && std::find(grids.begin(), grids.end(), gsz) == grids.end()) grids.push_back(gsz);
                    }
                    for (int gsz : grids) {
                        LevelChoice m = m0;
                        m.resident = gsz;
                        m.resident_g = groups;
                        m.resident_grid = true;
                        modes.push_back(m);
                    }
                }
            }
            if (cand.ncolours >= 4 && maxc <= 8 && schwarz_cluster_ok<V, T>(cand, maxc)) {
                LevelChoice m = m0;
                m.persist = maxc;
                m.staged = true;
                m.cluster = true;
                modes.push_back(m);
            }
            const char* force = std::getenv("AMGH_SMOOTHER_MODE");
            for (const LevelChoice& m : modes) {
                if (force && *force && std::string(force) != smoother_mode_name(m) &&
                    std::string(force) != smoother_mode_detail(m))
                    continue;
                if (m.resident > 0) schwarz_resident_prepare<V>(cand, m.resident, m.resident_g, s);
                set_smoother_mode(cand, m);
                float ms = 0.f;
                try {
                    ms = time_best_graph(s, 5, [&] {
                        if (cand.fused) {
                            launch_schwarz_fused<V, T>(cand, d.f.p, d.x.p, s);
                        } else if (cand.persist > 0) {
                            launch_schwarz_persistent<V, T>(cand, d.f.p, d.x.p, s);
                        } else {
                            for (int c : Engine::colour_sequence(cand.ncolours))
                                launch_schwarz_colourL<V, T>(cand, c, d.f.p, d.x.p, s);
                        }
                    });
                } catch (const CudaError& e) {
                    // a launch configuration the driver refuses (not a device fault): skip it
                    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
                    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                        cudaGraph_t g = nullptr;
                        cudaStreamEndCapture(s, &g);
                        if (g) cudaGraphDestroy(g);
                    }
                    cudaGetLastError();
                    if (cudaStreamSynchronize(s) != cudaSuccess) throw;
                    continue;
                }
                if (take_wait_flag(h, s)) {   // a bounded wait gave up: never choose this mode
                    cand.bar.zero(s);
                    continue;
                }
                if (ph.on)
                    std::fprintf(stderr, "[amgh] L%d tune lanes %2d %-22s %9.4f ms (%d steps)\n", l, Lc,
                                 smoother_mode_detail(m).c_str(), ms, 2 * cand.ncolours - 1);
                if (ms < best) {
                    best = ms;
                    const double kap = ch.kappa;
                    ch = m;
                    ch.kappa = kap;
                }
                if (smoother_mode_name(m) == "colour" && ms < best_colour) {
                    best_colour = ms;
                    colour_choice = m;
                }
            }
        }
        // plain per-colour launches (no waits between CTAs) unless another mode is clearly faster
        if (best_colour < 1e30f && best_colour <= 1.03f * best) {
            const double kap = ch.kappa;
            ch = colour_choice;
            ch.kappa = kap;
        }
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = ch;
    }
    build_smoother<V>(h, l, ch.L_sm, false, 0, false, d.sm, &d.col_nnz, &d.col_inv, &d.col_rows, s);
    // a mode whose shared-memory staging no longer fits (another device) falls back to per-colour
    // launches; the capacity queries also raise the kernels' shared-memory limits
    d.sm.persist = ch.persist;
    if (ch.cluster2 > 0 && !schwarz_cluster2_ok<V, T>(d.sm, ch.cluster2)) ch.cluster2 = 0;
    if (ch.resident > 0 && (ch.resident_grid ? (!cooperative_ok(h) ||
                                                schwarz_pipeline_cap<V, T>(d.sm, ch.resident_g) < ch.resident)
                                             : !schwarz_resident_ok<V, T>(d.sm, ch.resident, ch.resident_g)))
        ch.resident = 0;
    if (ch.resident > 0) schwarz_resident_prepare<V>(d.sm, ch.resident, ch.resident_g, s);
    if (ch.cluster && !schwarz_cluster_ok<V, T>(d.sm, ch.persist)) {
        ch.cluster = false;
        ch.staged = false;
        ch.persist = 0;
    }
    if (ch.staged && !ch.cluster && schwarz_staged_cap<V, T>(d.sm) < ch.persist) ch.staged = false;
    if (ch.stream > 0) ch.stream = std::min(ch.stream, schwarz_stream_cap<V, T>(d.sm, ch.stream_bufs));
    set_smoother_mode(d.sm, ch);
    ph.mark(s, "  smoother", l);
    AMGH_CUDA(cudaStreamSynchronize(s));
}

// storage precision of a level from the requested one and a condition estimate kappa of its
// smoother blocks: reduced precision with unit roundoff u only where kappa u <= 1/4, so that the
// block solves stay contractions; FP64 otherwise
static int level_precision(int requested, double kappa) {
    if (requested == AMGH_F64) return AMGH_F64;
    const double u32 = 5.9604644775390625e-08, u16 = 3.90625e-03;
    if (requested == AMGH_BF16 && kappa * u16 <= 0.25) return AMGH_BF16;
    if (kappa * u32 <= 0.25) return AMGH_F32;
    return AMGH_F64;
}

template <class T>
struct TypeTag {
    using type = T;
};

// the engine level of a storage precision, built on stream s
static void emplace_level(amgh_ctx* h, Engine* e, int l, LevelChoice& ch, cudaStream_t s) {
    auto make = [&](auto tag) {
        using Lv = typename decltype(tag)::type;
        e->L.emplace_back(std::in_place_type<Lv>);
        build_level(h, l, std::get<Lv>(e->L.back()), ch, s);
    };
    if (ch.prec == AMGH_F64) make(TypeTag<LevelX<double, double>>{});
    else if (ch.prec == AMGH_F32) make(TypeTag<LevelX<float, float>>{});
    else make(TypeTag<LevelX<bf16, float>>{});
}

static double level_kappa(amgh_ctx* h, int l, cudaStream_t s) {
    const StarLayout& st = h->hl[l].stars;
    DevArray<double> kap;
    kap.alloc(1);
    kap.zero(s);
    DevArray<int32_t> dsp, dsi;
    dsp.upload(st.star_ptr, s);
    dsi.upload(st.star_idx, s);
    launch_star_kappa(h->A64[l], st.nstars, dsp.p, dsi.p, kap.p, h->errflag.p, s);
    double k = 0.0;
    AMGH_CUDA(cudaMemcpyAsync(&k, kap.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    AMGH_CUDA(cudaStreamSynchronize(s));
    return k;
}

// W = P^T A of level l for the fused residual + restriction (Eq. tl's coarse right-hand side by
// associativity), by the same symbolic and numeric products as the Galerkin operator.  Tuned
// (fuse_restrict -1): Galerkin levels only.  On the finest level W is about as large as A (0.95
// of its entries on hex meshes), so the fused pass saves little there; on Galerkin levels W
// holds 0.04-0.5 of A's entries.
static bool wants_w(const amgh_params& prm, int l) { return prm.fuse_restrict > 0 || (prm.fuse_restrict < 0 && l > 0); }

static void form_w(amgh_ctx* h, int l, cudaStream_t s) {
    if (!wants_w(h->prm, l) || h->W64[l].nrows > 0) return;
    const DevCSR& PT = h->PT64[l];
    DevCSR Wd;
    if (!spgemm_symbolic(PT, h->A64[l], Wd, h->symflag.p, s)) {
        HostCSR hw = symbolic_product(h->hl[l].cz.PT, h->hl[l].A, 1);
        upload_csr(hw, Wd, s, false);
    }
    launch_ap_numeric(PT, h->A64[l], Wd, s);
    HostCSR wr;
    wr.nrows = Wd.nrows;
    wr.ncols = Wd.ncols;
    wr.ptr.resize(Wd.nrows + 1);
    AMGH_CUDA(cudaMemcpyAsync(wr.ptr.data(), Wd.ptr.p, sizeof(int32_t) * (Wd.nrows + 1), cudaMemcpyDeviceToHost, s));
    AMGH_CUDA(cudaStreamSynchronize(s));
    h->W64[l] = std::move(Wd);
    h->Wrows[l] = std::move(wr);
}

// the tuning-cache key level l will look up for the storage precision prec
static std::string level_key(amgh_ctx* h, int l, int prec) {
    const size_t vb = prec == AMGH_F64 ? sizeof(double) : prec == AMGH_F32 ? sizeof(float) : sizeof(bf16);
    return tune_key(h->hl[l], vb, vb, wants_w(h->prm, l) ? h->prm.fuse_restrict : 0);
}

// engine level l (its precision from the condition estimate, W, layouts, smoother), on stream s.
// With only_cached, a level whose launch choices are not cached yet is left alone (its tuning
// must time kernels without other work on the device): returns false then.
static bool build_engine_level(amgh_ctx* h, Engine* e, int l, cudaStream_t s, bool only_cached) {
    LevelChoice ch;
    // the condition estimate only decides a reduced precision; an FP64 request skips it
    ch.kappa = h->prm.precision == AMGH_F64 ? 0.0 : level_kappa(h, l, s);
    ch.prec = level_precision(h->prm.precision, ch.kappa);
    if (only_cached && tuning_enabled()) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        if (!g_tune_cache.count(level_key(h, l, ch.prec))) return false;
    }
    form_w(h, l, s);
    if ((int)e->choice.size() <= l) e->choice.resize(l + 1);
    e->choice[l] = ch;
    emplace_level(h, e, l, e->choice[l], s);
    return true;
}

// Builds the engine levels of a hierarchy while the setup loop coarsens further: level l is
// handed over once its P, P^T and smoother stars are final (an event on the setup stream), and
// built on the worker's own stream and host thread.  Only levels whose launch choices are cached
// are built here; the first level that would tune stops the worker, and the setup builds it and
// the rest afterwards, with nothing else running on the device.
struct EngineWorker {
    amgh_ctx* h;
    Engine* e;
    int dev = 0;
    cudaStream_t ws = nullptr;
    std::vector<cudaEvent_t> ev;
    std::mutex mu;
    std::condition_variable cv;
    int ready = 0;        // levels [0, ready) may be built
    bool closed = false;  // no further level will be handed over
    int built = 0;        // levels [0, built) were built here
    std::exception_ptr err;
    std::thread th;

    EngineWorker(amgh_ctx* hh, Engine* ee, int max_levels) : h(hh), e(ee), ev(max_levels, nullptr) {
        AMGH_CUDA(cudaGetDevice(&dev));
        AMGH_CUDA(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
        for (auto& x : ev) AMGH_CUDA(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
        th = std::thread([this] { run(); });
    }
    void run() {
        try {
            AMGH_CUDA(cudaSetDevice(dev));
            for (int l = 0;; ++l) {
                {
                    std::unique_lock<std::mutex> lock(mu);
                    cv.wait(lock, [&] { return ready > l || closed; });
                    if (ready <= l) return;
                }
                AMGH_CUDA(cudaStreamWaitEvent(ws, ev[l], 0));
                if (!build_engine_level(h, e, l, ws, true)) return;
                AMGH_CUDA(cudaStreamSynchronize(ws));
                built = l + 1;
            }
        } catch (...) {
            err = std::current_exception();
        }
    }
    // level l's inputs are enqueued on the setup stream s
    void hand_over(int l, cudaStream_t s) {
        AMGH_CUDA(cudaEventRecord(ev[l], s));
        {
            std::lock_guard<std::mutex> lock(mu);
            ready = l + 1;
        }
        cv.notify_one();
    }
    // waits for the worker; returns the number of levels it built
    int finish() {
        {
            std::lock_guard<std::mutex> lock(mu);
            closed = true;
        }
        cv.notify_one();
        if (th.joinable()) th.join();
        if (err) std::rethrow_exception(err);
        return built;
    }
    ~EngineWorker() {
        {
            std::lock_guard<std::mutex> lock(mu);
            closed = true;
        }
        cv.notify_one();
        if (th.joinable()) th.join();
        if (ws) {
            cudaStreamSynchronize(ws);
            cudaStreamDestroy(ws);
        }
        for (auto x : ev)
            if (x) cudaEventDestroy(x);
    }
};

static void build_engine(amgh_ctx* h, Engine* e, int from = 0) {
    cudaStream_t s = h->s;
    const int nlev = (int)h->hl.size();
    e->nlev = nlev;
    if (from == 0) {
        e->L.clear();
        e->choice.clear();
    }
    DevPhases ph;
    for (int l = from; l + 1 < nlev; ++l) {
        if (l > from) ph.mark(s, "engine level", l - 1);
        build_engine_level(h, e, l, s, false);
    }
    e->choice.resize(nlev);
    // coarsest level: dense inverse, precision from its 1-norm condition estimate
    const HostCSR& Ac = h->hl.back().A;
    const int nL = Ac.nrows;
    e->nL = nL;
    std::vector<double> inv((size_t)nL * nL);
    AMGH_CUDA(cudaMemcpyAsync(inv.data(), h->cinv64.p, sizeof(double) * inv.size(), cudaMemcpyDeviceToHost, s));
    AMGH_CUDA(cudaStreamSynchronize(s));
    double na = 0, ni = 0;
    for (int c = 0; c < nL; ++c) {
        double sa = 0, si = 0;
        for (int r = 0; r < nL; ++r) si += std::fabs(inv[(size_t)r * nL + c]);
        for (int32_t q = Ac.ptr[c]; q < Ac.ptr[c + 1]; ++q) sa += std::fabs(Ac.val[q]);   // symmetric
        na = std::max(na, sa);
        ni = std::max(ni, si);
    }
    LevelChoice& chL = e->choice[nlev - 1];
    chL.kappa = na * ni;
    chL.prec = level_precision(h->prm.precision, chL.kappa) == AMGH_F64 ? AMGH_F64 : AMGH_F32;
    if (chL.prec == AMGH_F64) {
        e->L.emplace_back(std::in_place_type<LevelX<double, double>>);
        auto& d = std::get<LevelX<double, double>>(e->L.back());
        d.n = nL;
        d.f.alloc(nL);
        d.x.alloc(nL);
        e->cinv_d.alloc((size_t)nL * nL);
        AMGH_CUDA(cudaMemcpyAsync(e->cinv_d.p, h->cinv64.p, sizeof(double) * inv.size(), cudaMemcpyDeviceToDevice, s));
    } else {
        e->L.emplace_back(std::in_place_type<LevelX<float, float>>);
        auto& d = std::get<LevelX<float, float>>(e->L.back());
        d.n = nL;
        d.f.alloc(nL);
        d.x.alloc(nL);
        e->cinv_f.alloc((size_t)nL * nL);
        launch_convert<float>(h->cinv64.p, e->cinv_f.p, (int64_t)nL * nL, s);
    }
    if (!e->level0_double()) {
        const int64_t n0 = h->hl[0].A.nrows;
        e->io_in.alloc(n0);
        e->io_out.alloc(n0);
    }
    AMGH_CUDA(cudaStreamSynchronize(s));
}

static void check_flag(amgh_ctx* h, const char* what) {
    int flag = 0;
    AMGH_CUDA(cudaMemcpyAsync(&flag, h->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    AMGH_CUDA(cudaStreamSynchronize(h->s));
    if (flag) throw StatusError{AMGH_ERR_NOT_SPD, std::string("non-positive pivot in ") + what};
}

static void check_csr_args(const amgh_csr* M) {
    if (!M || !M->row_ptr || (M->nnz > 0 && (!M->col || !M->val)))
        throw StatusError{AMGH_ERR_INVALID_ARG, "null CSR pointer"};
    if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0 || M->nrows >= INT32_MAX || M->ncols >= INT32_MAX ||
        M->nnz >= INT32_MAX)
        throw StatusError{AMGH_ERR_INVALID_ARG, "CSR dimensions out of range"};
}

static HostCSR to_host(const amgh_csr* M, cudaStream_t s, bool host_only = false) {
    check_csr_args(M);
    HostCSR h;
    h.nrows = (int)M->nrows;
    h.ncols = (int)M->ncols;
    const double t0 = now_ms();
    h.ptr.resize(h.nrows + 1);
    h.idx.resize(M->nnz);
    h.val.resize(M->nnz);
    const double t1 = now_ms();
    if (!M->on_device) {
        std::memcpy(h.ptr.data(), M->row_ptr, sizeof(int32_t) * (h.nrows + 1));
        if (M->nnz) {
            std::memcpy(h.idx.data(), M->col, sizeof(int32_t) * M->nnz);
            std::memcpy(h.val.data(), M->val, sizeof(double) * M->nnz);
        }
    } else {
        if (host_only) throw StatusError{AMGH_ERR_INVALID_ARG, "host CSR required"};
        AMGH_CUDA(cudaMemcpyAsync(h.ptr.data(), M->row_ptr, sizeof(int32_t) * (h.nrows + 1), cudaMemcpyDeviceToHost, s));
        if (M->nnz) {
            AMGH_CUDA(cudaMemcpyAsync(h.idx.data(), M->col, sizeof(int32_t) * M->nnz, cudaMemcpyDeviceToHost, s));
            AMGH_CUDA(cudaMemcpyAsync(h.val.data(), M->val, sizeof(double) * M->nnz, cudaMemcpyDeviceToHost, s));
        }
        AMGH_CUDA(cudaStreamSynchronize(s));
    }
    if (std::getenv("AMGH_VERBOSE"))
        std::fprintf(stderr, "[amgh]   input %lld x %lld, %lld nonzeros: allocate %.1f ms, copy %.1f ms\n",
                     (long long)M->nrows, (long long)M->ncols, (long long)M->nnz, t1 - t0, now_ms() - t1);
    if (h.ptr[h.nrows] != M->nnz) throw StatusError{AMGH_ERR_INVALID_ARG, "row_ptr[nrows] != nnz"};
    return h;
}

static void check_params(const amgh_params& prm) {
    if (prm.max_levels < 1 || prm.max_levels > 32 || prm.coarse_size < 1 || prm.ring < 1 || prm.p_max < 1 ||
        prm.p_max > 256 || prm.precision < 0 || prm.precision > 2 || !(prm.theta >= 0.0 && prm.theta <= 1.0) ||
        !(prm.stall_ratio > 0.0) || prm.dense_tail < 0 || prm.dense_tail > 16384)
        throw StatusError{AMGH_ERR_INVALID_ARG, "parameter out of range"};
    if (prm.interp != AMGH_INTERP_LOCAL && prm.interp != AMGH_INTERP_LEARNED && prm.interp != AMGH_INTERP_GEOMETRIC &&
        prm.interp != AMGH_INTERP_CONSTRAINED)
        throw StatusError{AMGH_ERR_INVALID_ARG, "unknown interpolation mode"};
    if (prm.coarsening != AMGH_COARSEN_ALGEBRAIC && prm.coarsening != AMGH_COARSEN_REFINEMENT)
        throw StatusError{AMGH_ERR_INVALID_ARG, "unknown coarsening mode"};
    if (prm.coarsening == AMGH_COARSEN_REFINEMENT && (prm.mesh_n < 4 || prm.mesh_n % 2))
        throw StatusError{AMGH_ERR_INVALID_ARG, "refinement coarsening needs mesh_n even and at least 4"};
    if (prm.interp == AMGH_INTERP_GEOMETRIC && prm.coarsening != AMGH_COARSEN_REFINEMENT)
        throw StatusError{AMGH_ERR_INVALID_ARG, "the geometric interpolation needs refinement coarsening"};
    if (prm.interp == AMGH_INTERP_LEARNED && !prm.mlp)
        throw StatusError{AMGH_ERR_INVALID_ARG, "learned interpolation needs a network (params.mlp)"};
}

static void check_inputs(const HostCSR& A, const HostCSR& G) {
    std::string e = check_csr(A, true);
    if (e.empty()) e = check_csr(G, false);
    if (e.empty() && G.nrows != A.nrows) e = "G must have as many rows as A";
    if (e.empty()) e = check_gradient(G);
    if (!e.empty()) throw StatusError{AMGH_ERR_INVALID_ARG, e};
    if (A.nrows == 0) throw StatusError{AMGH_ERR_INVALID_ARG, "empty system"};
}

static int host_threads() {
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = std::max(1, std::min(omp_get_max_threads(), 32));
#endif
    return nthreads;
}

static Params graph_params(const amgh_params& prm) {
    Params gp;
    gp.theta = prm.theta;
    gp.ring = prm.ring;
    gp.p_max = prm.p_max;
    return gp;
}

// level 0 graph steps only, on the host (structure-only handle)
static void host_structure_impl(amgh_ctx* h, const amgh_csr* Ain, const amgh_csr* Gin) {
    check_params(h->prm);
    HostCSR A = to_host(Ain, nullptr, true);
    HostCSR G = to_host(Gin, nullptr, true);
    check_inputs(A, G);
    h->structure_only = true;
    h->hl.emplace_back();
    LevelHost& cur = h->hl.back();
    cur.A = std::move(A);
    cur.G = std::move(G);
    std::string msg = h->prm.coarsening == AMGH_COARSEN_REFINEMENT
                          ? coarsen_level_refinement(cur.A, cur.G, h->prm.mesh_n,
                                                     h->prm.interp == AMGH_INTERP_GEOMETRIC, graph_params(h->prm),
                                                     cur.cz, host_threads())
                          : coarsen_level(cur.A, cur.G, graph_params(h->prm), cur.cz, host_threads());
    if (!msg.empty())
        throw StatusError{h->prm.coarsening == AMGH_COARSEN_REFINEMENT ? AMGH_ERR_INVALID_ARG : AMGH_ERR_SETUP_STALL, msg};
    if (cur.cz.edges.empty()) throw StatusError{AMGH_ERR_SETUP_STALL, "the finest level produced no coarse edge"};
    msg = build_stars(cur.A, cur.G, cur.stars);
    if (!msg.empty()) throw StatusError{AMGH_ERR_UNSUPPORTED, msg};
    if (h->prm.interp == AMGH_INTERP_CONSTRAINED) {
        CommutingRows crow;
        msg = commuting_rows(cur.G, cur.cz, crow, host_threads());
        if (!msg.empty()) throw StatusError{AMGH_ERR_UNSUPPORTED, msg};
        cur.Pn = std::move(crow.Pn);
    }
}

static void setup_impl(amgh_ctx* h, const amgh_csr* Ain, const amgh_csr* Gin) {
    DevPhases ph;
    cudaStream_t s = h->s;
    const auto& prm = h->prm;
    check_params(prm);
    // A goes to the device straight from the caller's arrays, before the host copy: from
    // page-locked arrays the transfer then runs while the host copies them
    check_csr_args(Ain);
    DevCSR dA;
    dA.nrows = (int)Ain->nrows;
    dA.ncols = (int)Ain->ncols;
    dA.nnz = Ain->nnz;
    dA.ptr.alloc(dA.nrows + 1);
    dA.idx.alloc(std::max<int64_t>(1, dA.nnz));
    dA.val.alloc(std::max<int64_t>(1, dA.nnz));
    {
        const cudaMemcpyKind k = Ain->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        AMGH_CUDA(cudaMemcpyAsync(dA.ptr.p, Ain->row_ptr, sizeof(int32_t) * (dA.nrows + 1), k, s));
        if (dA.nnz) {
            AMGH_CUDA(cudaMemcpyAsync(dA.idx.p, Ain->col, sizeof(int32_t) * dA.nnz, k, s));
            AMGH_CUDA(cudaMemcpyAsync(dA.val.p, Ain->val, sizeof(double) * dA.nnz, k, s));
        }
    }
    HostCSR A = to_host(Ain, s);
    HostCSR G = to_host(Gin, s);
    ph.mark(s, "inputs to host");
    check_inputs(A, G);
    ph.mark(s, "input checks");
    const int nthreads = host_threads();
    Params gp = graph_params(prm);
    h->errflag.alloc(1);
    h->errflag.zero(s);
    h->waitflag.alloc(1);
    h->waitflag.zero(s);
    h->symflag.alloc(1);
    gp.symbolic_galerkin = false;
    {
        int dev = 0;
        AMGH_CUDA(cudaGetDevice(&dev));
        AMGH_CUDA(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    // level arrays keep their addresses while the engine worker reads finished levels
    const size_t cap = (size_t)prm.max_levels + 1;
    h->hl.reserve(cap);
    h->A64.reserve(cap);
    h->P64.reserve(cap);
    h->PT64.reserve(cap);
    h->W64.reserve(cap);
    h->Wrows.reserve(cap);
    auto* e = new Engine();
    h->eng.reset(e);
    e->prof = &h->prof;
    std::unique_ptr<EngineWorker> worker;
    {
        const char* ov = std::getenv("AMGH_ENGINE_OVERLAP");
        if (!(ov && std::string(ov) == "0")) worker.reset(new EngineWorker(h, e, (int)cap));
    }
    const bool refine = prm.coarsening == AMGH_COARSEN_REFINEMENT;
    int mesh_n = prm.mesh_n;
    for (int l = 0;; ++l) {
        h->hl.emplace_back();
        LevelHost& cur = h->hl.back();
        cur.A = std::move(A);
        cur.G = std::move(G);
        h->A64.push_back(std::move(dA));
        const int n = cur.A.nrows;
        bool coarsest = n <= prm.coarse_size || l + 1 >= prm.max_levels;
        double t0 = now_ms();
        // refinement coarsening halves the mesh per level while it stays even
        if (refine && (mesh_n % 2 || mesh_n < 4)) coarsest = true;
        if (!coarsest) {
            std::string msg = refine ? coarsen_level_refinement(cur.A, cur.G, mesh_n,
                                                                prm.interp == AMGH_INTERP_GEOMETRIC, gp, cur.cz,
                                                                nthreads)
                                     : coarsen_level(cur.A, cur.G, gp, cur.cz, nthreads);
            if (!msg.empty()) throw StatusError{l == 0 && refine ? AMGH_ERR_INVALID_ARG : AMGH_ERR_SETUP_STALL, msg};
            const int nc = (int)cur.cz.edges.size();
            if (nc == 0 || (double)nc > prm.stall_ratio * n) {
                if (l == 0) throw StatusError{AMGH_ERR_SETUP_STALL, "the finest level produced no usable coarse level"};
                coarsest = true;
                cur.cz = Coarsening();
            }
        }
        h->host_ms += now_ms() - t0;
        ph.mark(s, "host graph steps", l);
        if (coarsest) break;
        t0 = now_ms();
        double t_stars = 0.0, t_comm = 0.0;
        Coarsening& cz = cur.cz;
        const int nc = (int)cz.edges.size();
        h->P64.emplace_back();
        h->PT64.emplace_back();
        DevCSR& P = h->P64.back();
        DevCSR& PT = h->PT64.back();
        // patterns from the host; values: zero, the exterior +-1 of R^T scattered on the device,
        // the interior filled below by the local solves (or the network)
        upload_csr(cz.P, P, s, false);
        upload_csr(cz.PT, PT, s, false);
        AMGH_CUDA(cudaMemsetAsync(P.val.p, 0, sizeof(double) * P.nnz, s));
        AMGH_CUDA(cudaMemsetAsync(PT.val.p, 0, sizeof(double) * PT.nnz, s));
        std::vector<int32_t> e4(4 * (size_t)nc);
        int maxp = 0;
        for (int c = 0; c < nc; ++c) {
            e4[4 * c] = cz.edges[c].d1;
            e4[4 * c + 1] = cz.edges[c].s1;
            e4[4 * c + 2] = cz.edges[c].d2;
            e4[4 * c + 3] = cz.edges[c].s2;
            maxp = std::max(maxp, cz.patch_ptr[c + 1] - cz.patch_ptr[c]);
        }
        h->max_patch.push_back(maxp);
        {
            DevArray<int32_t> de4, dpp, dpi;
            DevArray<int64_t> dpos, dpost;
            de4.upload(e4, s);
            dpp.upload(cz.patch_ptr, s);
            dpi.upload(cz.patch_idx, s);
            dpos.upload(cz.patch_pos_P, s);
            dpost.upload(cz.patch_pos_PT, s);
            {
                DevArray<int64_t> dex, dext;
                dex.upload(cz.ext_pos_P, s);
                dext.upload(cz.ext_pos_PT, s);
                launch_ext_scatter(nc, de4.p, dex.p, dext.p, P.val.p, PT.val.p, s);
                AMGH_CUDA(cudaStreamSynchronize(s));
            }
            // the finest P's fill time, on the stream, without a host synchronisation
            struct FillEvents {
                cudaEvent_t e0 = nullptr, e1 = nullptr;
                ~FillEvents() {
                    if (e0) cudaEventDestroy(e0);
                    if (e1) cudaEventDestroy(e1);
                }
            } fe;
            if (l == 0) {
                AMGH_CUDA(cudaEventCreate(&fe.e0));
                AMGH_CUDA(cudaEventCreate(&fe.e1));
                AMGH_CUDA(cudaEventRecord(fe.e0, s));
            }
            bool solved = false;
            auto* net = static_cast<amgh_mlp_ctx*>(prm.mlp);
            // per-row data of the commuting correction (interp CONSTRAINED), alive until the
            // flag check below has waited for its kernel
            CommutingRows crow;
            DevArray<int32_t> dcr_order, dcr_rows, dcr_nptr, dcr_comp, dcr_ptpos;
            DevArray<int16_t> dcr_ea, dcr_eb;
            DevArray<double> dcr_t;
            if (!cz.geo_ptr.empty()) {
                // the geometric interpolation: its weights are set, not solved for
                std::vector<double> pv(cz.P.nnz(), 0.0), ptv(cz.PT.nnz(), 0.0);
                for (int c = 0; c < nc; ++c) {
                    pv[cz.ext_pos_P[2 * (size_t)c]] = cz.edges[c].s1;
                    pv[cz.ext_pos_P[2 * (size_t)c + 1]] = cz.edges[c].s2;
                    ptv[cz.ext_pos_PT[2 * (size_t)c]] = cz.edges[c].s1;
                    ptv[cz.ext_pos_PT[2 * (size_t)c + 1]] = cz.edges[c].s2;
                }
                for (size_t q = 0; q < cz.geo_val.size(); ++q) {
                    pv[cz.patch_pos_P[q]] = cz.geo_val[q];
                    ptv[cz.patch_pos_PT[q]] = cz.geo_val[q];
                }
                AMGH_CUDA(cudaMemcpyAsync(P.val.p, pv.data(), sizeof(double) * pv.size(), cudaMemcpyHostToDevice, s));
                AMGH_CUDA(cudaMemcpyAsync(PT.val.p, ptv.data(), sizeof(double) * ptv.size(), cudaMemcpyHostToDevice, s));
                AMGH_CUDA(cudaStreamSynchronize(s));
                h->interp_used = AMGH_INTERP_GEOMETRIC;
            } else if (l == 0 && prm.interp == AMGH_INTERP_LEARNED && net && maxp <= MLP_SLOTS) {
                // the network predicts the interior values of every column of P on its patch
                DevArray<float> X, Y;
                X.alloc((size_t)nc * MLP_DIN);
                Y.alloc((size_t)nc * MLP_SLOTS);
                launch_mlp_features(h->A64[l], 0, nc, de4.p, dpp.p, dpi.p, nullptr, nullptr, X.p, nullptr, nullptr, s);
                AMGH_CUDA(cudaStreamSynchronize(s));
                AMGH_CUDA(cudaStreamSynchronize(net->s));
                mlp_forward(net->net, X.p, nc, Y.p, s);
                launch_mlp_scatter(0, nc, dpp.p, Y.p, dpos.p, dpost.p, P.val.p, PT.val.p, s);
                AMGH_CUDA(cudaStreamSynchronize(s));
                h->interp_used = AMGH_INTERP_LEARNED;
            } else {
                launch_patch_solve(h->A64[l], nc, de4.p, dpp.p, dpi.p, dpos.p, dpost.p, P.val.p, PT.val.p, maxp,
                                   h->errflag.p, s);
                solved = true;
            }
            // Eq. commuting (interp CONSTRAINED): the nodal interpolation and every interior row's
            // constraint are built on a helper thread while this one builds the smoother's stars
            // and the solves run; the device then corrects the rows
            const bool commute = solved && prm.interp == AMGH_INTERP_CONSTRAINED;
            // the finest P's fill time ends here, unless the correction still has to run
            if (l == 0 && !commute) AMGH_CUDA(cudaEventRecord(fe.e1, s));
            std::string comm_msg;
            std::vector<int32_t> order;
            int32_t cls_ptr[9] = {0};
            int sizes[8];
            const int ncls = commute_size_classes(sizes);
            struct Joiner {
                std::thread t;
                ~Joiner() {
                    if (t.joinable()) t.join();
                }
            } comm;
            if (commute)
                comm.t = std::thread([&] {
                    try {
                        comm_msg = commuting_rows(cur.G, cz, crow, nthreads);
                        if (comm_msg.empty() && crow.max_nodes > sizes[ncls - 1])
                            comm_msg = "a row of the commuting correction touches " + std::to_string(crow.max_nodes) +
                                       " coarse nodes (at most " + std::to_string(sizes[ncls - 1]) + ")";
                        if (!comm_msg.empty()) return;
                        // rows grouped by the size class of their local node count
                        order.reserve(crow.rows.size());
                        for (int c = 0; c < ncls; ++c) {
                            const int lo = c ? sizes[c - 1] : -1;
                            for (size_t r = 0; r < crow.rows.size(); ++r) {
                                const int mr = crow.node_ptr[r + 1] - crow.node_ptr[r];
                                if (mr > lo && mr <= sizes[c]) order.push_back((int32_t)r);
                            }
                            cls_ptr[c + 1] = (int32_t)order.size();
                        }
                    } catch (const std::exception& e) {
                        comm_msg = std::string("commuting correction: ") + e.what();
                    }
                });
            // the smoother's node stars and colouring are host work: built while the solves run
            {
                const double ts = now_ms();
                std::string msg = build_stars(cur.A, cur.G, cur.stars);
                t_stars = now_ms() - ts;
                h->host_ms += t_stars;
                if (!msg.empty()) {
                    if (comm.t.joinable()) comm.t.join();
                    throw StatusError{AMGH_ERR_UNSUPPORTED, msg};
                }
            }
            if (commute) {
                const double tc = now_ms();
                comm.t.join();
                if (!comm_msg.empty()) throw StatusError{AMGH_ERR_UNSUPPORTED, comm_msg};
                t_comm = now_ms() - tc;   // what the helper thread took beyond the stars
                h->host_ms += t_comm;
                dcr_order.upload(order, s);
                dcr_rows.upload(crow.rows, s);
                dcr_nptr.upload(crow.node_ptr, s);
                dcr_comp.upload(crow.comp, s);
                dcr_ptpos.upload(crow.pt_pos, s);
                dcr_ea.upload(crow.ea, s);
                dcr_eb.upload(crow.eb, s);
                dcr_t.upload(crow.t, s);
                launch_commute_rows(cls_ptr, dcr_order.p, dcr_rows.p, P.ptr.p, P.val.p, PT.val.p, dcr_ptpos.p,
                                    dcr_ea.p, dcr_eb.p, dcr_nptr.p, dcr_t.p, dcr_comp.p, h->errflag.p, s);
                h->interp_used = AMGH_INTERP_CONSTRAINED;
                cur.Pn = std::move(crow.Pn);
                if (l == 0) AMGH_CUDA(cudaEventRecord(fe.e1, s));
            }
            if (solved) check_flag(h, "a local harmonic-extension solve or the commuting correction");
            if (l == 0) {
                float ms = 0.f;
                AMGH_CUDA(cudaEventSynchronize(fe.e1));
                AMGH_CUDA(cudaEventElapsedTime(&ms, fe.e0, fe.e1));
                h->interp_ms = ms;
            }
        }
        ph.mark(s, "P upload + patch solves", l);
        // Galerkin product: symbolic patterns on the device (the host's when a row overflows the
        // kernel's set), then the numeric products with their fixed summation order
        DevCSR AP, Ac;
        if (!spgemm_symbolic(h->A64[l], P, AP, h->symflag.p, s)) {
            HostCSR hp = symbolic_product(cur.A, cz.P, nthreads);
            upload_csr(hp, AP, s, false);
        }
        launch_ap_numeric(h->A64[l], P, AP, s);
        if (!spgemm_symbolic(PT, AP, Ac, h->symflag.p, s)) {
            HostCSR hap;
            hap.nrows = AP.nrows;
            hap.ncols = AP.ncols;
            hap.ptr.resize(AP.nrows + 1);
            hap.idx.resize(AP.nnz);
            AMGH_CUDA(cudaMemcpyAsync(hap.ptr.data(), AP.ptr.p, sizeof(int32_t) * (AP.nrows + 1), cudaMemcpyDeviceToHost, s));
            AMGH_CUDA(cudaMemcpyAsync(hap.idx.data(), AP.idx.p, sizeof(int32_t) * AP.nnz, cudaMemcpyDeviceToHost, s));
            AMGH_CUDA(cudaStreamSynchronize(s));
            HostCSR hc = symbolic_product(cz.PT, hap, nthreads);
            upload_csr(hc, Ac, s, false);
        }
        launch_ac_numeric(PT, AP, Ac, s);
        // placeholders of W = P^T A, formed with the level's engine (form_w)
        h->W64.emplace_back();
        h->Wrows.emplace_back();
        HostCSR An;   // the next level's matrix, on the host for its graph steps
        An.nrows = Ac.nrows;
        An.ncols = Ac.ncols;
        An.ptr.resize(Ac.nrows + 1);
        An.idx.resize(Ac.nnz);
        An.val.resize(Ac.nnz);
        AMGH_CUDA(cudaMemcpyAsync(An.ptr.data(), Ac.ptr.p, sizeof(int32_t) * (Ac.nrows + 1), cudaMemcpyDeviceToHost, s));
        AMGH_CUDA(cudaMemcpyAsync(An.idx.data(), Ac.idx.p, sizeof(int32_t) * Ac.nnz, cudaMemcpyDeviceToHost, s));
        AMGH_CUDA(cudaMemcpyAsync(An.val.data(), Ac.val.p, sizeof(double) * Ac.nnz, cudaMemcpyDeviceToHost, s));
        AMGH_CUDA(cudaStreamSynchronize(s));
        if (worker) worker->hand_over(l, s);   // level l's P, P^T and stars are final
        if (refine) mesh_n /= 2;
        h->dev_ms += std::max(0.0, now_ms() - t0 - t_stars - t_comm);
        ph.mark(s, "Galerkin + download", l);
        A = std::move(An);
        G = cz.Gc;
        G.val = cz.Gc.val;
        dA = std::move(Ac);
    }
    const int nL = h->hl.back().A.nrows;
    if (nL > 2048) throw StatusError{AMGH_ERR_UNSUPPORTED, "coarsest level larger than 2048 DoFs"};
    double t0 = now_ms();
    {
        DevArray<double> work;
        work.alloc((size_t)nL * nL);
        h->cinv64.alloc((size_t)nL * nL);
        launch_coarse_inverse(h->A64.back(), h->cinv64.p, work.p, h->errflag.p, s);
        check_flag(h, "the coarsest factorisation");
    }
    ph.mark(s, "coarsest inverse");
    const int built = worker ? worker->finish() : 0;
    worker.reset();
    ph.mark(s, "engine levels built beside the setup loop");
    {
        // the sub-cycle below the first small level is linear in its right-hand side: apply it as
        // one dense operator, computed column block by column block with the multi-RHS V-cycle
        const int nlev = (int)h->hl.size();
        int t = -1;
        for (int l = 1; l + 1 < nlev && prm.dense_tail > 0; ++l)
            if (h->hl[l].A.nrows <= prm.dense_tail) { t = l; break; }
        auto build_tail = [h, t](cudaStream_t ts) {
            h->meng.reset(new MultiEngine());
            h->meng->build(h->hl, h->A64, h->P64, h->PT64, h->cinv64.p, h->errflag.p, ts, t);
            h->meng->dense_tail(t, h->dense_tail_B, ts);
            AMGH_CUDA(cudaStreamSynchronize(ts));
        };
        // The tail and the engine levels are independent: build the tail on its own stream and
        // thread meanwhile, unless the engine build times launch modes (the tail's kernels would
        // disturb those timings), i.e. only for FP64 storage with every level's choice cached
        bool overlap = t > 0 && prm.precision == AMGH_F64;
        if (overlap && tuning_enabled()) {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            for (int l = built; l + 1 < nlev && overlap; ++l) overlap = g_tune_cache.count(level_key(h, l, AMGH_F64)) > 0;
        }
        if (overlap) {
            int dev = 0;
            AMGH_CUDA(cudaGetDevice(&dev));
            cudaStream_t ts = nullptr;
            AMGH_CUDA(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
            std::exception_ptr tail_error;
            std::thread worker([&] {
                try {
                    AMGH_CUDA(cudaSetDevice(dev));
                    build_tail(ts);
                } catch (...) {
                    tail_error = std::current_exception();
                }
            });
            std::exception_ptr engine_error;
            try {
                build_engine(h, e, built);
            } catch (...) {
                engine_error = std::current_exception();
            }
            worker.join();
            cudaStreamDestroy(ts);
            if (engine_error) std::rethrow_exception(engine_error);
            if (tail_error) std::rethrow_exception(tail_error);
            ph.mark(s, "V-cycle engine + dense tail (concurrent)");
        } else {
            build_engine(h, e, built);
            ph.mark(s, "V-cycle engine");
            if (t > 0) build_tail(s);
        }
        if (t > 0) {
            check_flag(h, "a smoother block of the dense tail");
            h->dense_tail_level = t;
            e->tail = t;
            const int nt = h->hl[t].A.nrows;
            if (vectors_double(e->L[t])) {
                e->tail_d = std::move(h->dense_tail_B);   // FP64 level: the engine keeps the operator
            } else {
                e->tail_f.alloc((size_t)nt * nt);
                launch_convert<float>(h->dense_tail_B.p, e->tail_f.p, (int64_t)nt * nt, s);
            }
            AMGH_CUDA(cudaStreamSynchronize(s));
            h->dense_tail_B = DevArray<double>();
            ph.mark(s, "dense tail");
        }
    }
    check_flag(h, "a smoother block");
    build_sell<double>(h->hl[0].A, h->A64[0], h->A0, s);
    h->nnzA0 = h->hl[0].A.nnz();
    const int64_t n0 = h->hl[0].A.nrows;
    h->kp.alloc(n0);
    h->kq.alloc(n0);
    h->kro.alloc(n0);
    h->partial.alloc(2 * RED_BLOCKS);
    h->scal.alloc(S_COUNT);
    h->scal.zero(s);
    h->iter.alloc(1);
    h->iter.zero(s);
    AMGH_CUDA(cudaMallocHost(&h->hscal, sizeof(double) * S_COUNT));
    h->eng->capture(s);
    AMGH_CUDA(cudaStreamSynchronize(s));
    h->dev_ms += now_ms() - t0;
    ph.mark(s, "outer SpMV + graph capture");
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// device that owns a device pointer (-1 for host memory or an unknown pointer)
static int device_of(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? at.device : -1;
}

static double read_scalar(amgh_ctx* h, int slot) {
    AMGH_CUDA(cudaMemcpyAsync(h->hscal, h->scal.p, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, h->s));
    AMGH_CUDA(cudaStreamSynchronize(h->s));
    return h->hscal[slot];
}

// accumulate kernel timings after a stream sync: the V-cycle graph's event pairs (recorded by
// its last launch) and, for the outer SpMV class, the pairs recorded eagerly since the last call
static void harvest(amgh_ctx* h) {
    if (!h->prof.enabled) { h->vc_pending = false; return; }
    if (h->vc_pending) {
        // every V-cycle since the last harvest recorded its own pairs (pool entries [0, used))
        if (h->eng->prof_pairs) h->prof.harvest(h->prof.used);
        h->vc_pending = false;
    }
    if (h->prof.kind == K_SPMV) {
        if (h->prof.used) h->prof.harvest(h->prof.used);
        h->prof.used = 0;
    }
}

// V-cycle on the engine's FP64 buffers; profiling pairs are harvested by the caller after a sync
static void run_vcycle(amgh_ctx* h) {
    h->launches += h->eng->vcycle(h->s);
    h->vc_pending = true;
}

struct Staged {
    const double* f;
    double* x;
};

static Staged stage_in(amgh_ctx* h, const double* f, double* x, bool copy_x) {
    const int64_t n = h->hl[0].A.nrows;
    bool df = is_device_ptr(f), dx = is_device_ptr(x);
    if (df != dx) throw StatusError{AMGH_ERR_INVALID_ARG, "f and x must both be host or both be device pointers"};
    if (df) return {f, x};
    if (h->stage_f.n != (size_t)n) { h->stage_f.alloc(n); h->stage_x.alloc(n); }
    AMGH_CUDA(cudaMemcpyAsync(h->stage_f.p, f, sizeof(double) * n, cudaMemcpyHostToDevice, h->s));
    if (copy_x) AMGH_CUDA(cudaMemcpyAsync(h->stage_x.p, x, sizeof(double) * n, cudaMemcpyHostToDevice, h->s));
    return {h->stage_f.p, h->stage_x.p};
}

static void stage_out(amgh_ctx* h, const Staged& st, double* x) {
    const int64_t n = h->hl[0].A.nrows;
    if (st.x != x) AMGH_CUDA(cudaMemcpyAsync(x, st.x, sizeof(double) * n, cudaMemcpyDeviceToHost, h->s));
    AMGH_CUDA(cudaStreamSynchronize(h->s));
}

template <class F>
static void outer_spmv_timed(amgh_ctx* h, F&& fn) {
    if (h->prof.match(K_SPMV, 0)) {
        auto ev = h->prof.next();
        h->prof.bytes_used.resize(h->prof.used);
        h->prof.bytes_used[h->prof.used - 1] = (double)h->nnzA0 * 12.0 + 4.0 * h->A0.nrows + 16.0 * h->A0.nrows;
        h->prof.record(ev.first, h->s);
        fn();
        h->prof.record(ev.second, h->s);
    } else {
        fn();
    }
}

static amgh_status pcg_impl(amgh_ctx* h, const double* f_in, double* x_in, double tol, int maxit, int* iters,
                            double* relres) {
    if (maxit < 0 || !(tol >= 0.0)) throw StatusError{AMGH_ERR_INVALID_ARG, "bad tol or maxit"};
    cudaStream_t s = h->s;
    const int64_t n = h->hl[0].A.nrows;
    const bool flexible = h->prm.precision != AMGH_F64;
    Staged st = stage_in(h, f_in, x_in, true);
    const double* f = st.f;
    double* x = st.x;
    double* r = h->eng->in64();
    double* z = h->eng->out64();
    double* p = h->kp.p;
    double* q = h->kq.p;
    h->prof.used = 0;
    outer_spmv_timed(h, [&] { launch_sell<double, double>(SELL_RESID, h->A0, x, f, nullptr, r, s); });
    launch_dot(n, r, r, h->partial.p, s);
    launch_reduce(h->partial.p, RED_BLOCKS, h->scal.p, SC_STORE, s);
    h->launches += 3;
    const double r0 = std::sqrt(read_scalar(h, S_TMP));
    harvest(h);
    h->prof.used = 0;
    int it = 0;
    double rel = 0.0;
    amgh_status status = AMGH_OK;
    if (r0 > 0.0) {
        run_vcycle(h);
        launch_dot2(n, r, z, nullptr, h->partial.p, s);
        launch_reduce(h->partial.p, RED_BLOCKS, h->scal.p, SC_RZ, s);
        AMGH_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        h->launches += 2;
        rel = 1.0;
        bool conv = false;
        for (it = 1; it <= maxit; ++it) {
            outer_spmv_timed(h, [&] { launch_spmv_dot(h->A0, p, q, h->partial.p, s); });
            launch_reduce(h->partial.p, RED_BLOCKS, h->scal.p, SC_ALPHA, s);
            launch_cg_update(n, x, r, flexible ? h->kro.p : nullptr, p, q, h->scal.p, h->partial.p, s);
            launch_reduce(h->partial.p, RED_BLOCKS, h->scal.p, SC_STORE, s);
            h->launches += 4;
            const double rr = read_scalar(h, S_TMP);   // the V-cycles' event pairs wait for the end
            rel = std::sqrt(rr) / r0;
            if (!(rel == rel)) throw StatusError{AMGH_ERR_NOT_CONVERGED, "residual became NaN"};
            if (rel <= tol) { conv = true; break; }
            run_vcycle(h);
            launch_dot2(n, r, z, flexible ? h->kro.p : nullptr, h->partial.p, s);
            launch_reduce(h->partial.p, RED_BLOCKS, h->scal.p, flexible ? SC_BETA_FCG : SC_BETA_CG, s);
            launch_p_update(n, p, z, h->scal.p, s);
            h->launches += 3;
        }
        if (!conv) { it = maxit; status = AMGH_ERR_NOT_CONVERGED; }
    }
    stage_out(h, st, x_in);
    harvest(h);
    h->prof.used = 0;
    if (iters) *iters = it;
    if (relres) *relres = rel;
    if (status != AMGH_OK) h->err = "PCG reached maxit before the tolerance";
    return status;
}

// ---------------------------------------------------------------------------------------------
// Device-resident PCG: the whole solve is one branch of a CUDA graph.  The branch holds a
// prologue (r = f - A x, r0, the first iteration) and a WHILE node whose body runs one more
// iteration (z = B r, beta, p, q = A p, alpha, x and r, the stopping test that sets the node's
// condition).  No host round trip happens until the graph has finished.
// ---------------------------------------------------------------------------------------------
static void add_solve_branch(amgh_ctx* h, cudaGraph_t G, cudaStream_t cs, const double* f, double* x, double tol,
                             int maxit) {
    const int64_t n = h->hl[0].A.nrows;
    const bool flexible = h->prm.precision != AMGH_F64;
    double* r = h->eng->in64();
    double* z = h->eng->out64();
    double* p = h->kp.p;
    double* q = h->kq.p;
    double* ro = flexible ? h->kro.p : nullptr;
    cudaGraphConditionalHandle hw;
    AMGH_CUDA(cudaGraphConditionalHandleCreate(&hw, G, 1, cudaGraphCondAssignDefault));
    // event nodes are not allowed inside conditional bodies: the branch is never timed
    struct ProfOff {
        Profiler& p;
        bool was;
        ProfOff(Profiler& q) : p(q), was(q.enabled) { p.enabled = false; }
        ~ProfOff() { p.enabled = was; }
    } prof_off(h->prof);
    const int64_t before = launch_counter().load();
    AMGH_CUDA(cudaStreamBeginCaptureToGraph(cs, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    std::vector<cudaGraphNode_t> deps;
    int64_t pro = 0, body = 0;
    try {
        launch_sell<double, double>(SELL_RESID, h->A0, x, f, nullptr, r, cs);
        launch_dot(n, r, r, h->partial.p, cs);
        launch_reduce(h->partial.p, RED_BLOCKS, h->scal.p, SC_STORE, cs);
        launch_pcg_start(h->scal.p, h->iter.p, cs);
        pro += 4 + h->eng->enqueue(cs);
        launch_dot2(n, r, z, nullptr, h->partial.p, cs);
        launch_reduce(h->partial.p, RED_BLOCKS, h->scal.p, SC_RZ, cs);
        AMGH_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, cs));
        launch_spmv_dot(h->A0, p, q, h->partial.p, cs);
        launch_reduce(h->partial.p, RED_BLOCKS, h->scal.p, SC_ALPHA, cs);
        launch_cg_update(n, x, r, ro, p, q, h->scal.p, h->partial.p, cs);
        launch_reduce(h->partial.p, RED_BLOCKS, h->scal.p, SC_STORE, cs);
        launch_pcg_check(hw, h->scal.p, h->iter.p, tol, maxit, cs);
        pro += 7;
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t* d = nullptr;
        size_t nd = 0;
        AMGH_CUDA(cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &d, nullptr, &nd));
        deps.assign(d, d + nd);
    } catch (...) {
        cudaGraph_t g;
        cudaStreamEndCapture(cs, &g);
        launch_counter().store(before);
        throw;
    }
    cudaGraph_t g_out;
    AMGH_CUDA(cudaStreamEndCapture(cs, &g_out));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hw;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    AMGH_CUDA(cudaGraphAddNode(&wnode, G, deps.data(), nullptr, deps.size(), &cp));
    cudaGraph_t bg = cp.conditional.phGraph_out[0];
    AMGH_CUDA(cudaStreamBeginCaptureToGraph(cs, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
        body += h->eng->enqueue(cs);
        launch_dot2(n, r, z, ro, h->partial.p, cs);
        launch_reduce(h->partial.p, RED_BLOCKS, h->scal.p, flexible ? SC_BETA_FCG : SC_BETA_CG, cs);
        launch_p_update(n, p, z, h->scal.p, cs);
        launch_spmv_dot(h->A0, p, q, h->partial.p, cs);
        launch_reduce(h->partial.p, RED_BLOCKS, h->scal.p, SC_ALPHA, cs);
        launch_cg_update(n, x, r, ro, p, q, h->scal.p, h->partial.p, cs);
        launch_reduce(h->partial.p, RED_BLOCKS, h->scal.p, SC_STORE, cs);
        launch_pcg_check(hw, h->scal.p, h->iter.p, tol, maxit, cs);
        body += 8;
    } catch (...) {
        cudaGraph_t g;
        cudaStreamEndCapture(cs, &g);
        launch_counter().store(before);
        throw;
    }
    AMGH_CUDA(cudaStreamEndCapture(cs, &bg));
    launch_counter().store(before);
    h->s_pro_launches = pro;
    h->s_body_launches = body;
}

// read back (iterations, relres) of a finished device-resident solve
static void read_solve_result(amgh_ctx* h, int* it, double* rel) {
    int k = 0;
    AMGH_CUDA(cudaMemcpyAsync(&k, h->iter.p, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    AMGH_CUDA(cudaMemcpyAsync(h->hscal, h->scal.p, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, h->s));
    AMGH_CUDA(cudaStreamSynchronize(h->s));
    *it = k;
    *rel = h->hscal[S_REL];
    h->launches += h->s_pro_launches + (int64_t)std::max(0, k - 1) * h->s_body_launches;
    launch_counter().fetch_add(h->s_pro_launches + (int64_t)std::max(0, k - 1) * h->s_body_launches);
}

static amgh_status pcg_device_impl(amgh_ctx* h, const double* f_in, double* x_in, double tol, int maxit, int* iters,
                                   double* relres) {
    Staged st = stage_in(h, f_in, x_in, true);
    if (!h->sexec || h->s_f != st.f || h->s_x != st.x || h->s_tol != tol || h->s_maxit != maxit) {
        h->drop_solve_graph();
        AMGH_CUDA(cudaGraphCreate(&h->sgraph, 0));
        add_solve_branch(h, h->sgraph, h->s, st.f, st.x, tol, maxit);
        AMGH_CUDA(cudaGraphInstantiate(&h->sexec, h->sgraph, 0));
        h->s_f = st.f;
        h->s_x = st.x;
        h->s_tol = tol;
        h->s_maxit = maxit;
    }
    AMGH_CUDA(cudaGraphLaunch(h->sexec, h->s));
    int it = 0;
    double rel = 0.0;
    read_solve_result(h, &it, &rel);
    stage_out(h, st, x_in);
    if (!(rel == rel)) throw StatusError{AMGH_ERR_NOT_CONVERGED, "residual became NaN"};
    if (iters) *iters = it;
    if (relres) *relres = rel;
    if (rel > tol) {
        h->err = "PCG reached maxit before the tolerance";
        return AMGH_ERR_NOT_CONVERGED;
    }
    return AMGH_OK;
}

static amgh_status amg_impl(amgh_ctx* h, const double* f_in, double* x_in, double tol, int maxit, int* iters,
                            double* relres) {
    if (maxit < 0 || !(tol >= 0.0)) throw StatusError{AMGH_ERR_INVALID_ARG, "bad tol or maxit"};
    cudaStream_t s = h->s;
    const int64_t n = h->hl[0].A.nrows;
    Staged st = stage_in(h, f_in, x_in, true);
    double* r = h->eng->in64();
    double* z = h->eng->out64();
    h->prof.used = 0;
    double r0 = 0.0, rel = 0.0;
    int it = 0;
    amgh_status status = AMGH_OK;
    for (it = 0; it <= maxit; ++it) {
        outer_spmv_timed(h, [&] { launch_sell<double, double>(SELL_RESID, h->A0, st.x, st.f, nullptr, r, s); });
        launch_dot(n, r, r, h->partial.p, s);
        launch_reduce(h->partial.p, RED_BLOCKS, h->scal.p, SC_STORE, s);
        h->launches += 3;
        const double nr = std::sqrt(read_scalar(h, S_TMP));
        harvest(h);
        h->prof.used = 0;
        if (it == 0) r0 = nr;
        rel = r0 > 0 ? nr / r0 : 0.0;
        if (r0 == 0.0 || rel <= tol) break;
        if (it == maxit) { status = AMGH_ERR_NOT_CONVERGED; break; }
        run_vcycle(h);
        launch_axpy1(n, st.x, z, s);
        h->launches += 1;
    }
    stage_out(h, st, x_in);
    harvest(h);
    h->prof.used = 0;
    if (iters) *iters = it;
    if (relres) *relres = rel;
    if (status != AMGH_OK) h->err = "stand-alone V-cycle iteration reached maxit before the tolerance";
    return status;
}

}  // namespace amgh

namespace amgh {

// Host-driven PCG whose Krylov buffers come from the caller (see krylov_scratch.h).  It mirrors
// pcg_impl step for step; the V-cycle is enqueued kernel by kernel, so nothing is instantiated.
static amgh_status pcg_scratch_impl(amgh_ctx* h, const double* f, double* x, double tol, int maxit, int* iters,
                                    double* relres, const KrylovScratch& ks, int64_t max_rows) {
    if (maxit < 0 || !(tol >= 0.0)) throw StatusError{AMGH_ERR_INVALID_ARG, "bad tol or maxit"};
    const int64_t n = h->hl[0].A.nrows;
    if (n > max_rows)
        throw StatusError{AMGH_ERR_INVALID_ARG, "system has " + std::to_string(n) +
                                                    " rows; the allocation-free solve takes at most " +
                                                    std::to_string(max_rows)};
    if (!is_device_ptr(f) || !is_device_ptr(x))
        throw StatusError{AMGH_ERR_INVALID_ARG, "the allocation-free solve takes device pointers only"};
    int cur = -1;
    AMGH_CUDA(cudaGetDevice(&cur));
    if (cur != h->dev || device_of(f) != h->dev || device_of(x) != h->dev)
        throw StatusError{AMGH_ERR_INVALID_ARG, "the allocation-free solve needs the handle's device (" +
                                                    std::to_string(h->dev) + ") current and f, x on it"};
    struct ProfOff {
        Profiler& p;
        bool was;
        ProfOff(Profiler& q) : p(q), was(q.enabled) { p.enabled = false; }
        ~ProfOff() { p.enabled = was; }
    } prof_off(h->prof);
    cudaStream_t s = h->s;
    const bool flexible = h->prm.precision != AMGH_F64;
    double* r = h->eng->in64();
    double* z = h->eng->out64();
    auto read = [&](int slot) {   // into the handle's pinned scalars, as read_scalar does
        AMGH_CUDA(cudaMemcpyAsync(h->hscal, ks.scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s));
        AMGH_CUDA(cudaStreamSynchronize(s));
        return h->hscal[slot];
    };
    AMGH_CUDA(cudaMemsetAsync(ks.scal, 0, sizeof(double) * S_COUNT, s));   // shared scalars start at zero
    launch_sell<double, double>(SELL_RESID, h->A0, x, f, nullptr, r, s);
    launch_dot(n, r, r, ks.partial, s);
    launch_reduce(ks.partial, RED_BLOCKS, ks.scal, SC_STORE, s);
    const double r0 = std::sqrt(read(S_TMP));
    int it = 0;
    double rel = 0.0;
    amgh_status status = AMGH_OK;
    if (r0 > 0.0) {
        h->eng->enqueue(s);
        launch_dot2(n, r, z, nullptr, ks.partial, s);
        launch_reduce(ks.partial, RED_BLOCKS, ks.scal, SC_RZ, s);
        AMGH_CUDA(cudaMemcpyAsync(ks.p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        rel = 1.0;
        bool conv = false;
        for (it = 1; it <= maxit; ++it) {
            launch_spmv_dot(h->A0, ks.p, ks.q, ks.partial, s);
            launch_reduce(ks.partial, RED_BLOCKS, ks.scal, SC_ALPHA, s);
            launch_cg_update(n, x, r, flexible ? ks.r_old : nullptr, ks.p, ks.q, ks.scal, ks.partial, s);
            launch_reduce(ks.partial, RED_BLOCKS, ks.scal, SC_STORE, s);
            rel = std::sqrt(read(S_TMP)) / r0;
            if (!(rel == rel)) throw StatusError{AMGH_ERR_NOT_CONVERGED, "residual became NaN"};
            if (rel <= tol) { conv = true; break; }
            h->eng->enqueue(s);
            launch_dot2(n, r, z, flexible ? ks.r_old : nullptr, ks.partial, s);
            launch_reduce(ks.partial, RED_BLOCKS, ks.scal, flexible ? SC_BETA_FCG : SC_BETA_CG, s);
            launch_p_update(n, ks.p, z, ks.scal, s);
        }
        if (!conv) { it = maxit; status = AMGH_ERR_NOT_CONVERGED; }
    }
    AMGH_CUDA(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    if (relres) *relres = rel;
    if (status != AMGH_OK) h->err = "PCG reached maxit before the tolerance";
    return status;
}

}  // namespace amgh

namespace amgh {
// convergence factor of 10 stand-alone V-cycles on A x = 0 from x0 ~ U(-1,1) (probe stream, seed 0):
// (||r_10|| / ||r_0||)^(1/10)
static double measure_rho(amgh_ctx* h) {
    const int64_t n = h->hl[0].A.nrows;
    std::vector<double> x0(n), zero(n, 0.0);
    for (int64_t i = 0; i < n; ++i) x0[i] = 2.0 * splitmix_u01(STREAM_PROBE, 0, (uint64_t)i) - 1.0;
    DevArray<double> f, x;
    f.upload(zero, h->s);
    x.upload(x0, h->s);
    int it = 0;
    double rel = 0.0;
    amg_impl(h, f.p, x.p, 0.0, 10, &it, &rel);   // runs all 10 cycles and reports "not converged"
    h->err.clear();
    return it > 0 && rel > 0 ? std::pow(rel, 1.0 / it) : 0.0;
}

// storage of each level in the multi-RHS engine: FP64 for an FP64 request, else the single-system
// engine's choice from the level's condition estimate (FP32 where it chose FP32 or BF16)
static std::vector<int> multi_precisions(amgh_ctx* h) {
    std::vector<int> p(h->hl.size(), AMGH_F64);
    if (h->prm.precision == AMGH_F64 || !h->eng) return p;
    const auto* e = static_cast<const Engine*>(h->eng.get());
    for (size_t l = 0; l < p.size() && l < e->choice.size(); ++l)
        p[l] = e->choice[l].prec == AMGH_F64 ? AMGH_F64 : AMGH_F32;
    return p;
}

// the multi-RHS engine of the whole hierarchy (not the dense-tail one), built on first use
static MultiEngine& multi_engine(amgh_ctx* h) {
    if (!h->meng || h->meng->first_built > 0) {
        const std::vector<int> prec = multi_precisions(h);
        h->meng.reset(new MultiEngine());
        h->meng->build(h->hl, h->A64, h->P64, h->PT64, h->cinv64.p, h->errflag.p, h->s, 0, &prec);
    }
    return *h->meng;
}

static amgh_status pcg_multi_impl(amgh_ctx* h, const double* F_in, double* X_in, int k, double tol, int maxit,
                                  int* iters, double* relres) {
    if (k < 1 || k > 4096 || maxit < 0 || !(tol >= 0.0)) throw StatusError{AMGH_ERR_INVALID_ARG, "bad k, tol or maxit"};
    cudaStream_t s = h->s;
    const int64_t n = h->hl[0].A.nrows;
    const int KP = ((k + 31) / 32) * 32;
    MultiEngine& M = multi_engine(h);
    M.ensure_width(KP);
    // reduced-precision levels make the preconditioner inexact: flexible CG (Notay's FCG(1))
    const bool flexible = M.any_f32();
    const bool df = is_device_ptr(F_in), dx = is_device_ptr(X_in);
    if (df != dx) throw StatusError{AMGH_ERR_INVALID_ARG, "F and X must both be host or both be device pointers"};
    DevArray<double> Fs, Xs;
    const double* F = F_in;
    double* X = X_in;
    if (!df) {
        Fs.alloc((size_t)n * k);
        Xs.alloc((size_t)n * k);
        AMGH_CUDA(cudaMemcpyAsync(Fs.p, F_in, sizeof(double) * n * k, cudaMemcpyHostToDevice, s));
        AMGH_CUDA(cudaMemcpyAsync(Xs.p, X_in, sizeof(double) * n * k, cudaMemcpyHostToDevice, s));
        F = Fs.p;
        X = Xs.p;
    }
    DevArray<double> MF, MX, MP, MQ, alpha, beta, MR, MZ, MRold;
    MF.alloc((size_t)n * KP);
    MX.alloc((size_t)n * KP);
    MP.alloc((size_t)n * KP);
    MQ.alloc((size_t)n * KP);
    alpha.alloc(KP);
    beta.alloc(KP);
    // an FP64 level 0 reads its right-hand side from its F and leaves its result in its X; an FP32
    // one gets them converted
    double* R = M.L[0].F.p;
    double* Z = M.L[0].X.p;
    if (M.L[0].f32) {
        MR.alloc((size_t)n * KP);
        MZ.alloc((size_t)n * KP);
        R = MR.p;
        Z = MZ.p;
    }
    if (flexible) MRold.alloc((size_t)n * KP);
    auto precondition = [&] {
        M.load_rhs(R, s);
        M.vcycle_from(0, s);
        M.store_result(Z, s);
    };
    launch_to_rowmajor(F, n, k, KP, MF.p, s);
    launch_to_rowmajor(X, n, k, KP, MX.p, s);
    launch_spmm(MM_RESID, h->A64[0], KP, MX.p, MF.p, nullptr, R, s);
    std::vector<double> rr0(KP), rr(KP), rz(KP), rzn(KP), pq(KP), al(KP, 0.0), be(KP, 0.0);
    auto coldot = [&](const double* a, const double* b, std::vector<double>& out) {
        launch_coldot(a, b, n, KP, M.partial.p, M.colv.p, s);
        AMGH_CUDA(cudaMemcpyAsync(out.data(), M.colv.p, sizeof(double) * KP, cudaMemcpyDeviceToHost, s));
        AMGH_CUDA(cudaStreamSynchronize(s));
    };
    coldot(R, R, rr0);
    std::vector<char> active(KP, 0);
    std::vector<int> it_c(k, 0);
    std::vector<double> rel_c(k, 0.0);
    int nact = 0;
    for (int c = 0; c < k; ++c) {
        active[c] = rr0[c] > 0.0;
        nact += active[c];
    }
    std::vector<double> rzo(KP, 0.0);
    int it = 0;
    if (nact) {
        precondition();
        coldot(R, Z, rz);
        AMGH_CUDA(cudaMemcpyAsync(MP.p, Z, sizeof(double) * n * KP, cudaMemcpyDeviceToDevice, s));
        for (it = 1; it <= maxit && nact; ++it) {
            launch_spmm(MM_AX, h->A64[0], KP, MP.p, nullptr, nullptr, MQ.p, s);
            coldot(MP.p, MQ.p, pq);
            for (int c = 0; c < KP; ++c) al[c] = (active[c] && pq[c] != 0.0) ? rz[c] / pq[c] : 0.0;
            AMGH_CUDA(cudaMemcpyAsync(alpha.p, al.data(), sizeof(double) * KP, cudaMemcpyHostToDevice, s));
            launch_mcg_update(n, KP, MX.p, R, flexible ? MRold.p : nullptr, MP.p, MQ.p, alpha.p, s);
            coldot(R, R, rr);
            for (int c = 0; c < k; ++c) {
                if (!active[c]) continue;
                const double rel = std::sqrt(rr[c] / rr0[c]);
                it_c[c] = it;
                rel_c[c] = rel;
                if (!(rel == rel)) throw StatusError{AMGH_ERR_NOT_CONVERGED, "residual became NaN"};
                if (rel <= tol) { active[c] = 0; nact--; }
            }
            if (!nact) break;
            precondition();
            coldot(R, Z, rzn);
            // FCG(1): beta = <z_new, r_new - r_old> / <z_old, r_old>
            if (flexible) coldot(MRold.p, Z, rzo);
            for (int c = 0; c < KP; ++c) {
                const double num = flexible ? rzn[c] - rzo[c] : rzn[c];
                be[c] = active[c] && rz[c] != 0.0 ? num / rz[c] : 0.0;
                rz[c] = rzn[c];
            }
            AMGH_CUDA(cudaMemcpyAsync(beta.p, be.data(), sizeof(double) * KP, cudaMemcpyHostToDevice, s));
            launch_mp_update(n, KP, MP.p, Z, beta.p, s);
        }
    }
    launch_to_colmajor(MX.p, n, k, KP, X, s);
    if (!df) AMGH_CUDA(cudaMemcpyAsync(X_in, X, sizeof(double) * n * k, cudaMemcpyDeviceToHost, s));
    AMGH_CUDA(cudaStreamSynchronize(s));
    bool all = true;
    for (int c = 0; c < k; ++c) {
        if (iters) iters[c] = it_c[c];
        if (relres) relres[c] = rel_c[c];
        if (rr0[c] > 0.0 && rel_c[c] > tol) all = false;
    }
    if (!all) {
        h->err = "a right-hand side reached maxit before the tolerance";
        return AMGH_ERR_NOT_CONVERGED;
    }
    return AMGH_OK;
}

}  // namespace amgh

// =============================================================================================
// C-ABI
// =============================================================================================
template <class F>
static amgh_status guarded(amgh_ctx* h, F&& fn) {
    try {
        return fn();
    } catch (const StatusError& e) {
        if (h) h->err = e.msg;
        else g_setup_error = e.msg;
        return e.st;
    } catch (const CudaError& e) {
        std::string m = std::string("CUDA error ") + cudaGetErrorString(e.code) + " in " + e.where;
        if (h) h->err = m;
        else g_setup_error = m;
        return AMGH_ERR_CUDA;
    } catch (const std::bad_alloc&) {
        if (h) h->err = "host allocation failed";
        else g_setup_error = "host allocation failed";
        return AMGH_ERR_OOM;
    } catch (const std::exception& e) {
        if (h) h->err = e.what();
        else g_setup_error = e.what();
        return AMGH_ERR_INVALID_ARG;
    }
}

template <class F>
static amgh_status mlp_guarded(amgh_mlp m, F&& fn) {
    try {
        return fn();
    } catch (const StatusError& e) {
        m->err = e.msg;
        return e.st;
    } catch (const CudaError& e) {
        m->err = std::string("CUDA error ") + cudaGetErrorString(e.code) + " in " + e.where;
        return AMGH_ERR_CUDA;
    } catch (const std::bad_alloc&) {
        m->err = "host allocation failed";
        return AMGH_ERR_OOM;
    }
}

extern "C" {

void amgh_default_params(amgh_params* p) {
    if (!p) return;
    p->max_levels = 20;
    p->coarse_size = 100;
    p->precision = AMGH_F64;
    p->interp = AMGH_INTERP_LOCAL;
    p->ring = 1;
    p->p_max = 128;
    p->theta = 0.25;
    p->stall_ratio = 0.9;
    p->stream = nullptr;
    p->dense_tail = 8192;
    p->mlp = nullptr;
    p->rho_ref = 0.0;
    p->fuse_restrict = 0;
    p->coarsening = AMGH_COARSEN_ALGEBRAIC;
    p->mesh_n = 0;
}

amgh_status amgh_batch_setup(int nsys, const amgh_csr* A, const amgh_csr* G, const amgh_params* params,
                             amgh_handle* out) {
    if (nsys < 1 || !A || !G || !out) {
        g_setup_error = "batch setup needs nsys >= 1 and non-null arrays";
        return AMGH_ERR_INVALID_ARG;
    }
    for (int i = 0; i < nsys; ++i) out[i] = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        g_setup_error = "no usable current CUDA device";
        return AMGH_ERR_CUDA;
    }
    // a few setups at a time, each on its own host thread and stream; their host graph steps
    // split the host's cores between them
    const int conc = std::min(nsys, 4);
    int cores = 1;
#ifdef _OPENMP
    cores = omp_get_max_threads();
#endif
    const int per = std::max(1, cores / conc);
    std::atomic<int> next{0};
    std::vector<amgh_status> st(nsys, AMGH_OK);
    std::vector<std::string> msg(nsys);
    auto work = [&] {
        if (cudaSetDevice(dev) != cudaSuccess) {
            cudaGetLastError();
            for (int i; (i = next++) < nsys;) {
                st[i] = AMGH_ERR_CUDA;
                msg[i] = "cudaSetDevice failed on a batch thread";
            }
            return;
        }
#ifdef _OPENMP
        omp_set_num_threads(per);
#endif
        for (int i; (i = next++) < nsys;) {
            st[i] = amgh_setup(&A[i], &G[i], params, &out[i]);
            if (st[i] != AMGH_OK) msg[i] = g_setup_error;
        }
    };
    std::vector<std::thread> pool;
    try {
        for (int t = 1; t < conc; ++t) pool.emplace_back(work);
    } catch (...) {
    }
    work();
    for (auto& t : pool) t.join();
    for (int i = 0; i < nsys; ++i)
        if (st[i] != AMGH_OK) {
            for (int j = 0; j < nsys; ++j) {
                amgh_destroy(out[j]);
                out[j] = nullptr;
            }
            g_setup_error = "system " + std::to_string(i) + ": " + msg[i];
            return st[i];
        }
    return AMGH_OK;
}

amgh_status amgh_setup(const amgh_csr* A, const amgh_csr* G, const amgh_params* params, amgh_handle* out) {
    if (!out) return AMGH_ERR_INVALID_ARG;
    *out = nullptr;
    amgh_ctx* h = nullptr;
    try {
        h = new amgh_ctx();
    } catch (...) {
        g_setup_error = "host allocation failed";
        return AMGH_ERR_OOM;
    }
    if (params) h->prm = *params;
    else amgh_default_params(&h->prm);
    h->s = (cudaStream_t)h->prm.stream;
    amgh_status st = guarded(h, [&] {
        if (!h->s) {
            // a blocking stream of our own: ordered with the legacy default stream, capturable
            AMGH_CUDA(cudaStreamCreate(&h->s));
            h->own_stream = true;
        }
        AMGH_CUDA(cudaGetDevice(&h->dev));
        setup_impl(h, A, G);
        return AMGH_OK;
    });
    if (st == AMGH_ERR_NOT_SPD && h->interp_used == AMGH_INTERP_LEARNED) {
        // a predicted P whose coarse levels lost definiteness: the exact local solves instead
        amgh_params pe = h->prm;
        pe.interp = AMGH_INTERP_LOCAL;
        pe.mlp = nullptr;
        delete h;
        return amgh_setup(A, G, &pe, out);
    }
    if (st != AMGH_OK) {
        g_setup_error = h->err;
        delete h;
        return st;
    }
    if (h->interp_used == AMGH_INTERP_LEARNED) {
        // keep the learned interpolation only while its measured convergence factor stays within
        // 10% of the exact local solves' (a stored reference, or an exact setup measured here)
        st = guarded(h, [&] {
            h->rho_used = measure_rho(h);
            return AMGH_OK;
        });
        double rho_ex = h->prm.rho_ref;
        amgh_ctx* ex = nullptr;
        if (st == AMGH_OK && !(rho_ex > 0.0)) {
            amgh_params pe = h->prm;
            pe.interp = AMGH_INTERP_LOCAL;
            pe.mlp = nullptr;
            amgh_handle eh = nullptr;
            st = amgh_setup(A, G, &pe, &eh);
            ex = eh;
            if (st == AMGH_OK) {
                st = guarded(ex, [&] {
                    rho_ex = measure_rho(ex);
                    return AMGH_OK;
                });
            }
        }
        if (st != AMGH_OK) {
            g_setup_error = ex ? ex->err : h->err;
            delete ex;
            delete h;
            return st;
        }
        h->rho_exact = rho_ex;
        if (h->rho_used > 1.1 * rho_ex) {
            if (!ex) {
                amgh_params pe = h->prm;
                pe.interp = AMGH_INTERP_LOCAL;
                pe.mlp = nullptr;
                amgh_handle eh = nullptr;
                st = amgh_setup(A, G, &pe, &eh);
                if (st != AMGH_OK) {
                    delete h;
                    return st;
                }
                ex = eh;
                ex->rho_used = measure_rho(ex);
            } else {
                ex->rho_used = rho_ex;
            }
            ex->rho_exact = rho_ex;
            ex->interp_used = AMGH_INTERP_LOCAL;
            delete h;
            *out = ex;
            return AMGH_OK;
        }
        delete ex;
    }
    *out = h;
    return AMGH_OK;
}

amgh_status amgh_setup_host_structure(const amgh_csr* A, const amgh_csr* G, const amgh_params* params,
                                      amgh_handle* out) {
    if (!out) return AMGH_ERR_INVALID_ARG;
    *out = nullptr;
    amgh_ctx* h = nullptr;
    try {
        h = new amgh_ctx();
    } catch (...) {
        g_setup_error = "host allocation failed";
        return AMGH_ERR_OOM;
    }
    if (params) h->prm = *params;
    else amgh_default_params(&h->prm);
    amgh_status st = guarded(h, [&] {
        host_structure_impl(h, A, G);
        return AMGH_OK;
    });
    if (st != AMGH_OK) {
        g_setup_error = h->err;
        delete h;
        return st;
    }
    *out = h;
    return AMGH_OK;
}

amgh_status amgh_vcycle(amgh_handle h, const double* r, double* z) {
    if (!h || !r || !z || h->structure_only) return AMGH_ERR_INVALID_ARG;
    return guarded(h, [&] {
        const int64_t n = h->hl[0].A.nrows;
        bool dr = is_device_ptr(r), dz = is_device_ptr(z);
        if (dr != dz) throw StatusError{AMGH_ERR_INVALID_ARG, "r and z must both be host or both be device pointers"};
        auto kind_in = dr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        auto kind_out = dr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        h->prof.used = 0;
        AMGH_CUDA(cudaMemcpyAsync(h->eng->in64(), r, sizeof(double) * n, kind_in, h->s));
        run_vcycle(h);
        AMGH_CUDA(cudaMemcpyAsync(z, h->eng->out64(), sizeof(double) * n, kind_out, h->s));
        AMGH_CUDA(cudaStreamSynchronize(h->s));
        harvest(h);
        h->prof.used = 0;
        check_wait(h);
        return AMGH_OK;
    });
}

amgh_status amgh_pcg_solve(amgh_handle h, const double* f, double* x, double tol, int maxit, int* iters,
                           double* relres) {
    if (!h || !f || !x || h->structure_only) return AMGH_ERR_INVALID_ARG;
    return guarded(h, [&] {
        if (maxit < 0 || !(tol >= 0.0)) throw StatusError{AMGH_ERR_INVALID_ARG, "bad tol or maxit"};
        // kernel timing needs the host-driven loop (event nodes cannot sit in conditional bodies)
        const amgh_status st = (h->prof.enabled || maxit < 1 || h->host_loop)
                                   ? pcg_impl(h, f, x, tol, maxit, iters, relres)
                                   : pcg_device_impl(h, f, x, tol, maxit, iters, relres);
        check_wait(h);
        return st;
    });
}

amgh_status amgh_batch_pcg_solve(int nsys, const amgh_handle* hs, const double* const* f, double* const* x,
                                 double tol, int maxit, int* iters, double* relres) {
    if (nsys < 1 || !hs || !f || !x) return AMGH_ERR_INVALID_ARG;
    for (int i = 0; i < nsys; ++i)
        if (!hs[i] || hs[i]->structure_only || !f[i] || !x[i]) return AMGH_ERR_INVALID_ARG;
    amgh_ctx* h0 = hs[0];
    cudaGraph_t G = nullptr;
    cudaGraphExec_t GE = nullptr;
    amgh_status st = guarded(h0, [&] {
        if (maxit < 1 || !(tol >= 0.0)) throw StatusError{AMGH_ERR_INVALID_ARG, "bad tol or maxit"};
        for (int i = 0; i < nsys; ++i)
            if (!is_device_ptr(f[i]) || !is_device_ptr(x[i]))
                throw StatusError{AMGH_ERR_INVALID_ARG, "batched solves take device pointers"};
        AMGH_CUDA(cudaStreamSynchronize(h0->s));
        AMGH_CUDA(cudaGraphCreate(&G, 0));
        for (int i = 0; i < nsys; ++i) {
            if (i > 0) AMGH_CUDA(cudaStreamSynchronize(hs[i]->s));
            add_solve_branch(hs[i], G, h0->s, f[i], x[i], tol, maxit);   // independent branches
        }
        AMGH_CUDA(cudaGraphInstantiate(&GE, G, 0));
        AMGH_CUDA(cudaGraphLaunch(GE, h0->s));
        AMGH_CUDA(cudaStreamSynchronize(h0->s));
        for (int i = 0; i < nsys; ++i) check_wait(hs[i]);
        amgh_status all = AMGH_OK;
        for (int i = 0; i < nsys; ++i) {
            int it = 0;
            double rel = 0.0;
            read_solve_result(hs[i], &it, &rel);
            if (iters) iters[i] = it;
            if (relres) relres[i] = rel;
            if (!(rel <= tol)) all = AMGH_ERR_NOT_CONVERGED;
        }
        if (all != AMGH_OK) h0->err = "a system of the batch reached maxit before the tolerance";
        return all;
    });
    if (GE) cudaGraphExecDestroy(GE);
    if (G) cudaGraphDestroy(G);
    return st;
}

amgh_status amgh_amg_solve(amgh_handle h, const double* f, double* x, double tol, int maxit, int* iters,
                           double* relres) {
    if (!h || !f || !x || h->structure_only) return AMGH_ERR_INVALID_ARG;
    return guarded(h, [&] {
        const amgh_status st = amg_impl(h, f, x, tol, maxit, iters, relres);
        check_wait(h);
        return st;
    });
}

amgh_status amgh_pcg_solve_multi(amgh_handle h, const double* F, double* X, int k, double tol, int maxit, int* iters,
                                 double* relres) {
    if (!h || !F || !X || h->structure_only) return AMGH_ERR_INVALID_ARG;
    return guarded(h, [&] { return pcg_multi_impl(h, F, X, k, tol, maxit, iters, relres); });
}

amgh_status amgh_vcycle_multi(amgh_handle h, const double* Rin, double* Zout, int k) {
    if (!h || !Rin || !Zout || h->structure_only || k < 1 || k > 4096) return AMGH_ERR_INVALID_ARG;
    return guarded(h, [&] {
        if (!is_device_ptr(Rin) || !is_device_ptr(Zout))
            throw StatusError{AMGH_ERR_INVALID_ARG, "multi-RHS V-cycle takes device pointers"};
        cudaStream_t s = h->s;
        const int64_t n = h->hl[0].A.nrows;
        const int KP = ((k + 31) / 32) * 32;
        MultiEngine& M = multi_engine(h);
        M.ensure_width(KP);
        if (M.L[0].f32) {
            DevArray<double> tmp;
            tmp.alloc((size_t)n * KP);
            launch_to_rowmajor(Rin, n, k, KP, tmp.p, s);
            M.load_rhs(tmp.p, s);
            M.vcycle_from(0, s);
            M.store_result(tmp.p, s);
            launch_to_colmajor(tmp.p, n, k, KP, Zout, s);
        } else {
            launch_to_rowmajor(Rin, n, k, KP, M.L[0].F.p, s);
            M.vcycle_from(0, s);
            launch_to_colmajor(M.L[0].X.p, n, k, KP, Zout, s);
        }
        AMGH_CUDA(cudaStreamSynchronize(s));
        return AMGH_OK;
    });
}

amgh_status amgh_info(amgh_handle h, amgh_hier_info* info) {
    if (!h || !info || h->structure_only) return AMGH_ERR_INVALID_ARG;
    return guarded(h, [&] {
        std::memset(info, 0, sizeof(*info));
        const int nlev = (int)h->hl.size();
        info->levels = nlev;
        double nnz0 = (double)h->hl[0].A.nnz(), n0 = (double)h->hl[0].A.nrows, so = 0, sg = 0;
        for (int l = 0; l < nlev && l < 32; ++l) {
            const auto& L = h->hl[l];
            info->n[l] = L.A.nrows;
            info->nnz[l] = L.A.nnz();
            info->nnz_p[l] = L.cz.P.nnz();
            info->ncolours[l] = L.stars.ncolours;
            info->max_block[l] = L.stars.max_block;
            info->max_patch[l] = l < (int)h->max_patch.size() ? h->max_patch[l] : 0;
            so += L.A.nnz();
            sg += L.A.nrows;
        }
        info->op_complexity = so / nnz0;
        info->grid_complexity = sg / n0;
        info->setup_host_ms = h->host_ms;
        info->setup_device_ms = h->dev_ms;
        auto* e = static_cast<Engine*>(h->eng.get());
        info->dense_tail = h->dense_tail_level;
        info->interp_used = h->interp_used;
        info->rho = h->rho_used;
        info->rho_exact = h->rho_exact;
        info->interp_ms = h->interp_ms;
        for (int l = 0; l < nlev && l < 32 && l < (int)e->choice.size(); ++l) {
            info->precision[l] = e->choice[l].prec;
            info->lanes[l] = e->choice[l].L_sm;
            const LevelChoice& cl = e->choice[l];
            info->fused[l] = cl.fused ? 1 : cl.resident > 0 ? (cl.resident_grid ? 9 : 8) : cl.cluster2 > 0 ? 7
                           : cl.persist > 0 ? (cl.cluster ? 5 : cl.staged ? 3 : 2) : cl.stream > 0 ? 4
                           : cl.pdl ? 6 : 0;
            info->block_kappa[l] = e->choice[l].kappa;
            info->fused_rr[l] = cl.fuse_rr && l + 1 < nlev && (e->tail < 0 || l < e->tail) ? 1 : 0;
        }
        return AMGH_OK;
    });
}

amgh_status amgh_level_structure(amgh_handle h, int l, int64_t* n_nodes_aug, int64_t* n_edges,
                                 int64_t* n_coarse_nodes, int64_t* patch_nnz, int64_t* n_stars, int8_t* cf_state,
                                 int32_t* coarse_edges, int32_t* coarse_nodes, int32_t* patch_ptr, int32_t* patch_idx,
                                 int32_t* colour) {
    if (!h || l < 0 || l >= (int)h->hl.size() || (!h->structure_only && l + 1 >= (int)h->hl.size()))
        return AMGH_ERR_INVALID_ARG;
    return guarded(h, [&] {
        const auto& L = h->hl[l];
        const auto& cz = L.cz;
        if (n_nodes_aug) *n_nodes_aug = (int64_t)cz.state.size();
        if (n_edges) *n_edges = (int64_t)cz.edges.size();
        if (n_coarse_nodes) *n_coarse_nodes = (int64_t)cz.coarse_nodes.size();
        if (patch_nnz) *patch_nnz = (int64_t)cz.patch_idx.size();
        if (n_stars) *n_stars = L.stars.nstars;
        if (cf_state) std::memcpy(cf_state, cz.state.data(), cz.state.size());
        if (coarse_edges)
            for (size_t c = 0; c < cz.edges.size(); ++c) {
                const auto& e = cz.edges[c];
                int32_t v[7] = {e.d1, e.s1, e.d2, e.s2, e.i, e.k, e.j};
                std::memcpy(coarse_edges + 7 * c, v, sizeof(v));
            }
        if (coarse_nodes) std::memcpy(coarse_nodes, cz.coarse_nodes.data(), cz.coarse_nodes.size() * 4);
        if (patch_ptr) std::memcpy(patch_ptr, cz.patch_ptr.data(), cz.patch_ptr.size() * 4);
        if (patch_idx) std::memcpy(patch_idx, cz.patch_idx.data(), cz.patch_idx.size() * 4);
        if (colour) std::memcpy(colour, L.stars.colour.data(), L.stars.colour.size() * 4);
        return AMGH_OK;
    });
}

amgh_status amgh_level_matrix(amgh_handle h, int l, int which, int64_t* nrows, int64_t* ncols, int64_t* nnz,
                              int32_t* row_ptr, int32_t* col, double* val) {
    if (!h || l < 0 || l >= (int)h->hl.size() || which < 0 || which > 4) return AMGH_ERR_INVALID_ARG;
    const bool has_coarse = h->structure_only || l + 1 < (int)h->hl.size();
    if ((which == 1 || which == 3) && !has_coarse) return AMGH_ERR_INVALID_ARG;
    if (which == 4 && h->hl[l].Pn.ptr.empty()) return AMGH_ERR_INVALID_ARG;
    return guarded(h, [&] {
        const auto& L = h->hl[l];
        const HostCSR& M = which == 0 ? L.A
                           : which == 1 ? L.cz.P
                           : which == 2 ? L.G
                           : which == 4 ? L.Pn
                           : (h->structure_only ? L.cz.Ac : h->hl[l + 1].A);
        if (nrows) *nrows = M.nrows;
        if (ncols) *ncols = M.ncols;
        if (nnz) *nnz = M.nnz();
        if (row_ptr) std::memcpy(row_ptr, M.ptr.data(), M.ptr.size() * 4);
        if (col) std::memcpy(col, M.idx.data(), M.idx.size() * 4);
        if (val) {
            if (which == 2 || which == 4 || (h->structure_only && which != 3)) {
                std::memcpy(val, M.val.data(), M.val.size() * 8);
            } else if (h->structure_only) {
                std::memset(val, 0, sizeof(double) * M.nnz());
            } else {
                const DevCSR& D = which == 0 ? h->A64[l] : (which == 1 ? h->P64[l] : h->A64[l + 1]);
                AMGH_CUDA(cudaMemcpyAsync(val, D.val.p, sizeof(double) * D.nnz, cudaMemcpyDeviceToHost, h->s));
                AMGH_CUDA(cudaStreamSynchronize(h->s));
            }
        }
        return AMGH_OK;
    });
}

amgh_status amgh_level_apply(amgh_handle h, int l, int op, const double* f, const double* x, double* y) {
    if (!h || !x || !y || h->structure_only) return AMGH_ERR_INVALID_ARG;
    if ((op == 1 || op == 2 || op == 3) && !f) return AMGH_ERR_INVALID_ARG;
    return guarded(h, [&] {
        const bool was = h->prof.enabled;
        h->prof.enabled = false;   // single steps are never timed
        try {
            h->eng->level_apply(l, op, f, x, y, h->s);
        } catch (...) {
            h->prof.enabled = was;
            throw;
        }
        h->prof.enabled = was;
        AMGH_CUDA(cudaStreamSynchronize(h->s));
        check_wait(h);
        return AMGH_OK;
    });
}

amgh_status amgh_profile(amgh_handle h, int enable, int kind, int level) {
    if (!h || kind < 0 || kind > 7 || level < 0 || h->structure_only) return AMGH_ERR_INVALID_ARG;
    return guarded(h, [&] {
        h->prof.enabled = enable != 0;
        h->prof.gen++;
        h->prof.kind = kind;
        h->prof.level = level;
        h->prof.launches = 0;
        h->prof.total_ms = 0;
        h->prof.bytes = 0;
        h->prof.used = 0;
        return AMGH_OK;
    });
}

amgh_status amgh_kernel_stats(amgh_handle h, int64_t* launches, double* total_ms, double* algorithmic_bytes) {
    if (!h) return AMGH_ERR_INVALID_ARG;
    if (launches) *launches = h->prof.launches;
    if (total_ms) *total_ms = h->prof.total_ms;
    if (algorithmic_bytes) *algorithmic_bytes = h->prof.bytes;
    return AMGH_OK;
}

int64_t amgh_launch_count(amgh_handle) { return launch_counter().load(); }

amgh_status amgh_mlp_create(uint64_t seed, amgh_mlp* out) {
    if (!out) return AMGH_ERR_INVALID_ARG;
    *out = nullptr;
    auto* m = new (std::nothrow) amgh_mlp_ctx();
    if (!m) return AMGH_ERR_OOM;
    try {
        AMGH_CUDA(cudaStreamCreate(&m->s));
        mlp_init(m->net, seed, m->s);
        AMGH_CUDA(cudaStreamSynchronize(m->s));
    } catch (const CudaError& e) {
        g_setup_error = std::string("CUDA error ") + cudaGetErrorString(e.code) + " in " + e.where;
        delete m;
        return AMGH_ERR_CUDA;
    }
    *out = m;
    return AMGH_OK;
}

amgh_status amgh_mlp_add_samples(amgh_mlp m, amgh_handle h) {
    if (!m || !h || h->structure_only || h->hl.size() < 2) return AMGH_ERR_INVALID_ARG;
    amgh_status st = guarded(h, [&] {
        if (h->interp_used != AMGH_INTERP_LOCAL)
            throw StatusError{AMGH_ERR_INVALID_ARG, "samples come from a hierarchy built with exact local solves"};
        const Coarsening& cz = h->hl[0].cz;
        const int nc = (int)cz.edges.size();
        int maxp = 0;
        std::vector<int32_t> e4(4 * (size_t)nc);
        for (int c = 0; c < nc; ++c) {
            e4[4 * c] = cz.edges[c].d1;
            e4[4 * c + 1] = cz.edges[c].s1;
            e4[4 * c + 2] = cz.edges[c].d2;
            e4[4 * c + 3] = cz.edges[c].s2;
            maxp = std::max(maxp, cz.patch_ptr[c + 1] - cz.patch_ptr[c]);
        }
        if (maxp > MLP_SLOTS) throw StatusError{AMGH_ERR_UNSUPPORTED, "patches larger than the network's 64 slots"};
        cudaStream_t s = h->s;
        DevArray<int32_t> de4, dpp, dpi;
        DevArray<int64_t> dpos;
        de4.upload(e4, s);
        dpp.upload(cz.patch_ptr, s);
        dpi.upload(cz.patch_idx, s);
        dpos.upload(cz.patch_pos_P, s);
        AMGH_CUDA(cudaStreamSynchronize(m->s));
        MlpNet& net = m->net;
        mlp_reserve(net, net.nsamples + nc, s);
        launch_mlp_features(h->A64[0], 0, nc, de4.p, dpp.p, dpi.p, h->P64[0].val.p, dpos.p,
                            net.X.p + net.nsamples * MLP_DIN, net.T.p + net.nsamples * MLP_SLOTS,
                            net.M.p + net.nsamples * MLP_SLOTS, s);
        AMGH_CUDA(cudaStreamSynchronize(s));
        net.nsamples += nc;
        return AMGH_OK;
    });
    if (st != AMGH_OK) m->err = h->err;
    return st;
}

int64_t amgh_mlp_num_samples(amgh_mlp m) { return m ? m->net.nsamples : 0; }

amgh_status amgh_mlp_train(amgh_mlp m, int epochs, int batch, double lr, uint64_t seed, double* final_loss) {
    if (!m || epochs < 0 || batch < 1 || !(lr > 0)) return AMGH_ERR_INVALID_ARG;
    return mlp_guarded(m, [&] {
        double L = 0.0;
        for (int e = 0; e < epochs; ++e) L = mlp_epoch(m->net, batch, (float)lr, seed + (uint64_t)e, m->s);
        if (final_loss) *final_loss = L;
        return AMGH_OK;
    });
}

amgh_status amgh_mlp_set_precision(amgh_mlp m, int precision) {
    if (!m || (precision != AMGH_F32 && precision != AMGH_BF16)) return AMGH_ERR_INVALID_ARG;
    return mlp_guarded(m, [&] {
        m->net.bf16 = precision == AMGH_BF16;
        return AMGH_OK;
    });
}

amgh_status amgh_mlp_params(amgh_mlp m, float* out, float* in, int64_t* count) {
    if (!m) return AMGH_ERR_INVALID_ARG;
    return mlp_guarded(m, [&] {
        const int64_t n = m->net.count();
        if (count) *count = n;
        if (in) AMGH_CUDA(cudaMemcpyAsync(m->net.params.p, in, sizeof(float) * n, cudaMemcpyHostToDevice, m->s));
        if (out) AMGH_CUDA(cudaMemcpyAsync(out, m->net.params.p, sizeof(float) * n, cudaMemcpyDeviceToHost, m->s));
        AMGH_CUDA(cudaStreamSynchronize(m->s));
        return AMGH_OK;
    });
}

amgh_status amgh_mlp_loss_grad(amgh_mlp m, const float* X, const float* T, const float* M, int nb, double* loss,
                               float* grad) {
    if (!m || !X || !T || !M || nb < 1) return AMGH_ERR_INVALID_ARG;
    return mlp_guarded(m, [&] {
        cudaStream_t s = m->s;
        MlpNet& net = m->net;
        DevArray<float> dX, dT, dM;
        dX.upload(X, (size_t)nb * net.d_in, s);
        dT.upload(T, (size_t)nb * net.d_out, s);
        dM.upload(M, (size_t)nb * net.d_out, s);
        const double L = mlp_loss_grad(net, dX.p, dT.p, dM.p, nb, s);
        if (loss) *loss = L;
        if (grad) AMGH_CUDA(cudaMemcpyAsync(grad, net.grads.p, sizeof(float) * net.count(), cudaMemcpyDeviceToHost, s));
        AMGH_CUDA(cudaStreamSynchronize(s));
        return AMGH_OK;
    });
}

amgh_status amgh_mlp_predict(amgh_mlp m, const float* X, int64_t n, float* Y) {
    if (!m || !X || !Y || n < 0) return AMGH_ERR_INVALID_ARG;
    return mlp_guarded(m, [&] {
        cudaStream_t s = m->s;
        DevArray<float> dX, dY;
        dX.upload(X, (size_t)n * m->net.d_in, s);
        dY.alloc((size_t)n * m->net.d_out);
        mlp_forward(m->net, dX.p, n, dY.p, s);
        AMGH_CUDA(cudaMemcpyAsync(Y, dY.p, sizeof(float) * n * m->net.d_out, cudaMemcpyDeviceToHost, s));
        AMGH_CUDA(cudaStreamSynchronize(s));
        return AMGH_OK;
    });
}

amgh_status amgh_mlp_features(amgh_handle h, float* X, float* T, float* M, int64_t* n) {
    if (!h || h->structure_only || h->hl.size() < 2) return AMGH_ERR_INVALID_ARG;
    return guarded(h, [&] {
        const Coarsening& cz = h->hl[0].cz;
        const int nc = (int)cz.edges.size();
        if (n) *n = nc;
        if (!X && !T && !M) return AMGH_OK;
        cudaStream_t s = h->s;
        std::vector<int32_t> e4(4 * (size_t)nc);
        for (int c = 0; c < nc; ++c) {
            e4[4 * c] = cz.edges[c].d1;
            e4[4 * c + 1] = cz.edges[c].s1;
            e4[4 * c + 2] = cz.edges[c].d2;
            e4[4 * c + 3] = cz.edges[c].s2;
            if (cz.patch_ptr[c + 1] - cz.patch_ptr[c] > MLP_SLOTS)
                throw StatusError{AMGH_ERR_UNSUPPORTED, "patches larger than the network's 64 slots"};
        }
        DevArray<int32_t> de4, dpp, dpi;
        DevArray<int64_t> dpos;
        de4.upload(e4, s);
        dpp.upload(cz.patch_ptr, s);
        dpi.upload(cz.patch_idx, s);
        dpos.upload(cz.patch_pos_P, s);
        DevArray<float> dX, dT, dM;
        dX.alloc((size_t)nc * MLP_DIN);
        dT.alloc((size_t)nc * MLP_SLOTS);
        dM.alloc((size_t)nc * MLP_SLOTS);
        launch_mlp_features(h->A64[0], 0, nc, de4.p, dpp.p, dpi.p, h->P64[0].val.p, dpos.p, dX.p, dT.p, dM.p, s);
        if (X) AMGH_CUDA(cudaMemcpyAsync(X, dX.p, sizeof(float) * dX.n, cudaMemcpyDeviceToHost, s));
        if (T) AMGH_CUDA(cudaMemcpyAsync(T, dT.p, sizeof(float) * dT.n, cudaMemcpyDeviceToHost, s));
        if (M) AMGH_CUDA(cudaMemcpyAsync(M, dM.p, sizeof(float) * dM.n, cudaMemcpyDeviceToHost, s));
        AMGH_CUDA(cudaStreamSynchronize(s));
        return AMGH_OK;
    });
}

amgh_status amgh_selftest_wait_timeout(double* seconds) {
    try {
        cudaStream_t s = nullptr;
        AMGH_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        DevArray<int> err;
        err.alloc(1);
        const double t0 = now_ms();
        const bool fired = run_wait_timeout_probe(err.p, s);
        const double t1 = now_ms();
        cudaStreamDestroy(s);
        if (seconds) *seconds = (t1 - t0) / 1000.0;
        if (!fired) {
            g_setup_error = "the bounded wait did not report giving up";
            return AMGH_ERR_INVALID_ARG;
        }
        g_setup_error = "a device-side wait gave up (expected by this self-test)";
        return AMGH_ERR_TIMEOUT;
    } catch (const CudaError& e) {
        g_setup_error = std::string("CUDA error ") + cudaGetErrorString(e.code) + " in " + e.where;
        return AMGH_ERR_CUDA;
    }
}

const char* amgh_mlp_last_error(amgh_mlp m) { return m ? m->err.c_str() : g_setup_error.c_str(); }

void amgh_mlp_destroy(amgh_mlp m) { delete m; }

const char* amgh_last_error(amgh_handle h) {
    if (!h) return g_setup_error.c_str();
    return h->err.c_str();
}

void amgh_destroy(amgh_handle h) {
    if (!h) return;
    if (!h->structure_only) cudaStreamSynchronize(h->s);
    delete h;
}

}  // extern "C"

namespace amgh {

amgh_status fail_with(amgh_handle h, amgh_status st, const char* msg) {
    if (h && msg) h->err = msg;
    return st;
}

amgh_status pcg_with_scratch(amgh_handle h, const double* f, double* x, double tol, int maxit, int* iters,
                             double* relres, const KrylovScratch& ks, int64_t max_rows) {
    if (!h || !f || !x || h->structure_only) return AMGH_ERR_INVALID_ARG;
    return guarded(h, [&] {
        const amgh_status st = pcg_scratch_impl(h, f, x, tol, maxit, iters, relres, ks, max_rows);
        check_wait(h);
        return st;
    });
}

}  // namespace amgh
