// Host graph steps of the algebraic H(curl) coarsening (Section 4): Alg. 1 (augment G),
// the nodal graph of the dual operator and Alg. 2 (nodal C/F splitting), Alg. 3 (pairing fine
// edges along distance-two nodal paths), Eq. Gc (coarse gradient), the patches of the local
// interior harmonic extension (Eq. sparseP), the symbolic Galerkin patterns, and the node-star
// blocks and colouring of the OSS-l1 smoother (Section 5).
#include "host_graph.h"

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <numeric>
#include <utility>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace amgh {

namespace {

// phase timings on stderr when AMGH_VERBOSE=1
struct PhaseClock {
    bool on;
    std::chrono::steady_clock::time_point t;
    PhaseClock() : on(std::getenv("AMGH_VERBOSE") && std::getenv("AMGH_VERBOSE")[0] == '1'), t(std::chrono::steady_clock::now()) {}
    void mark(const char* what) {
        if (!on) return;
        auto now = std::chrono::steady_clock::now();
        std::fprintf(stderr, "[amgh] %-28s %8.1f ms\n", what, std::chrono::duration<double, std::milli>(now - t).count());
        t = now;
    }
};

inline int thread_id() {
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

inline int omp_threads() {
#ifdef _OPENMP
    return omp_get_num_threads();
#else
    return 1;
#endif
}

inline bool has(const HostCSR& M, int r, int c) {
    auto b = M.idx.begin() + M.ptr[r], e = M.idx.begin() + M.ptr[r + 1];
    return std::binary_search(b, e, c);
}

// Symbolic product row by row: out row r = union over t in X row r of Y row X.idx[t].
HostCSR symbolic_rows(const HostCSR& X, const HostCSR& Y, int nthreads) {
    HostCSR M;
    M.nrows = X.nrows;
    M.ncols = Y.ncols;
    M.ptr.assign(X.nrows + 1, 0);
    std::vector<std::vector<int32_t>> mark(nthreads, std::vector<int32_t>(Y.ncols, -1));
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
    for (int r = 0; r < X.nrows; ++r) {
        auto& mk = mark[thread_id()];
        int32_t cnt = 0;
        for (int32_t t = X.ptr[r]; t < X.ptr[r + 1]; ++t) {
            int32_t y = X.idx[t];
            for (int32_t u = Y.ptr[y]; u < Y.ptr[y + 1]; ++u) {
                int32_t c = Y.idx[u];
                if (mk[c] != r) { mk[c] = r; ++cnt; }
            }
        }
        M.ptr[r + 1] = cnt;
    }
    for (int r = 0; r < X.nrows; ++r) M.ptr[r + 1] += M.ptr[r];
    M.idx.resize(M.ptr[X.nrows]);
    for (auto& mk : mark) std::fill(mk.begin(), mk.end(), -1);
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
    for (int r = 0; r < X.nrows; ++r) {
        auto& mk = mark[thread_id()];
        int32_t pos = M.ptr[r];
        for (int32_t t = X.ptr[r]; t < X.ptr[r + 1]; ++t) {
            int32_t y = X.idx[t];
            for (int32_t u = Y.ptr[y]; u < Y.ptr[y + 1]; ++u) {
                int32_t c = Y.idx[u];
                if (mk[c] != r) { mk[c] = r; M.idx[pos++] = c; }
            }
        }
        std::sort(M.idx.begin() + M.ptr[r], M.idx.begin() + M.ptr[r + 1]);
    }
    return M;
}

}  // namespace

HostCSR symbolic_product(const HostCSR& X, const HostCSR& Y, int nthreads) { return symbolic_rows(X, Y, nthreads); }

HostCSR transpose_pattern(const HostCSR& M, bool with_values) {
    HostCSR T;
    T.nrows = M.ncols;
    T.ncols = M.nrows;
    T.ptr.assign(T.nrows + 1, 0);
    for (int32_t c : M.idx) T.ptr[c + 1]++;
    for (int r = 0; r < T.nrows; ++r) T.ptr[r + 1] += T.ptr[r];
    T.idx.resize(M.idx.size());
    if (with_values) T.val.resize(M.idx.size());
    std::vector<int32_t> cur(T.ptr.begin(), T.ptr.end() - 1);
    for (int r = 0; r < M.nrows; ++r)
        for (int32_t e = M.ptr[r]; e < M.ptr[r + 1]; ++e) {
            int32_t p = cur[M.idx[e]]++;
            T.idx[p] = r;
            if (with_values) T.val[p] = M.val[e];
        }
    return T;
}

// The same transpose in parallel: column counts with relaxed atomic adds, a scatter through atomic
// cursors, then each output row sorted by source row, which restores the sequential order
// (entries of one column come from distinct rows).  Small matrices take the sequential path.
HostCSR transpose_pattern(const HostCSR& M, bool with_values, int nthreads) {
    if (nthreads <= 1 || M.idx.size() < (size_t)(1 << 18)) return transpose_pattern(M, with_values);
    HostCSR T;
    T.nrows = M.ncols;
    T.ncols = M.nrows;
    T.ptr.assign(T.nrows + 1, 0);
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int r = 0; r < M.nrows; ++r)
        for (int32_t e = M.ptr[r]; e < M.ptr[r + 1]; ++e) __atomic_fetch_add(&T.ptr[M.idx[e] + 1], 1, __ATOMIC_RELAXED);
    for (int r = 0; r < T.nrows; ++r) T.ptr[r + 1] += T.ptr[r];
    T.idx.resize(M.idx.size());
    if (with_values) T.val.resize(M.idx.size());
    std::vector<int32_t> cur(T.ptr.begin(), T.ptr.end() - 1);
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int r = 0; r < M.nrows; ++r)
        for (int32_t e = M.ptr[r]; e < M.ptr[r + 1]; ++e) {
            const int32_t p = __atomic_fetch_add(&cur[M.idx[e]], 1, __ATOMIC_RELAXED);
            T.idx[p] = r;
            if (with_values) T.val[p] = M.val[e];
        }
#pragma omp parallel num_threads(nthreads)
    {
        std::vector<std::pair<int32_t, double>> row;
#pragma omp for schedule(dynamic, 4096)
        for (int c = 0; c < T.nrows; ++c) {
            const int32_t b = T.ptr[c], e = T.ptr[c + 1];
            if (!with_values) {
                std::sort(T.idx.begin() + b, T.idx.begin() + e);
                continue;
            }
            row.clear();
            for (int32_t q = b; q < e; ++q) row.push_back({T.idx[q], T.val[q]});
            std::sort(row.begin(), row.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
            for (int32_t q = b; q < e; ++q) {
                T.idx[q] = row[q - b].first;
                T.val[q] = row[q - b].second;
            }
        }
    }
    return T;
}

static std::string csr_row_error(const HostCSR& M, int r) {
    if (M.ptr[r + 1] < M.ptr[r]) return "row_ptr not monotone";
    if ((int64_t)M.ptr[r + 1] > (int64_t)M.idx.size()) return "row_ptr beyond nnz";
    for (int32_t e = M.ptr[r]; e < M.ptr[r + 1]; ++e) {
        const int32_t c = M.idx[e];
        if (c < 0 || c >= M.ncols) return "column index out of range in row " + std::to_string(r);
        if (e > M.ptr[r] && M.idx[e - 1] >= c) return "columns not strictly ascending in row " + std::to_string(r);
    }
    return "";
}

// the first failing row is found in parallel and then described
std::string check_csr(const HostCSR& M, bool square) {
    if (M.nrows < 0 || M.ncols < 0) return "negative dimension";
    if (square && M.nrows != M.ncols) return "matrix is not square";
    if ((int64_t)M.ptr.size() != (int64_t)M.nrows + 1 || M.ptr[0] != 0) return "bad row_ptr";
    int bad = INT32_MAX;
#pragma omp parallel for schedule(static) reduction(min : bad)
    for (int r = 0; r < M.nrows; ++r) {
        if (M.ptr[r + 1] < M.ptr[r] || (int64_t)M.ptr[r + 1] > (int64_t)M.idx.size()) {
            bad = std::min(bad, r);
            continue;
        }
        for (int32_t e = M.ptr[r]; e < M.ptr[r + 1]; ++e) {
            const int32_t c = M.idx[e];
            if (c < 0 || c >= M.ncols || (e > M.ptr[r] && M.idx[e - 1] >= c)) {
                bad = std::min(bad, r);
                break;
            }
        }
    }
    return bad == INT32_MAX ? std::string() : csr_row_error(M, bad);
}

static std::string gradient_row_error(const HostCSR& G, int r) {
    const int32_t n = G.ptr[r + 1] - G.ptr[r];
    // 0 entries: an interior edge joining two boundary nodes (e.g. a corner diagonal)
    if (n > 2) return "G row " + std::to_string(r) + " has " + std::to_string(n) + " entries (at most 2)";
    for (int32_t e = G.ptr[r]; e < G.ptr[r + 1]; ++e)
        if (G.val[e] != 1.0 && G.val[e] != -1.0) return "G entry other than +-1 in row " + std::to_string(r);
    if (n == 2 && G.val[G.ptr[r]] == G.val[G.ptr[r] + 1]) return "G row " + std::to_string(r) + " entries share a sign";
    return "";
}

std::string check_gradient(const HostCSR& G) {
    int bad = INT32_MAX;
#pragma omp parallel for schedule(static) reduction(min : bad)
    for (int r = 0; r < G.nrows; ++r)
        if (!gradient_row_error(G, r).empty()) bad = std::min(bad, r);
    return bad == INT32_MAX ? std::string() : gradient_row_error(G, bad);
}

// -------------------------------------------------------------------------------------------
// Alg. 1: one artificial column per boundary edge-row (a row of G with one entry delta; the
// new column holds -delta in that row).
// -------------------------------------------------------------------------------------------
static HostCSR augment(const HostCSR& G, int& nB, int nthreads) {
    const int n = G.nrows;
    HostCSR Gt;
    Gt.nrows = n;
    // boundary rows before row r: the artificial column of boundary row r is ncols + bpre[r]
    std::vector<int32_t> bpre(n + 1, 0);
    for (int r = 0; r < n; ++r) bpre[r + 1] = bpre[r] + (G.ptr[r + 1] - G.ptr[r] == 1);
    nB = bpre[n];
    Gt.ncols = G.ncols + nB;
    Gt.ptr.resize(n + 1);
    Gt.idx.resize(G.nnz() + nB);
    Gt.val.resize(G.nnz() + nB);
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int r = 0; r <= n; ++r) Gt.ptr[r] = G.ptr[r] + bpre[r];
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int r = 0; r < n; ++r) {
        int32_t o = Gt.ptr[r];
        for (int32_t e = G.ptr[r]; e < G.ptr[r + 1]; ++e, ++o) {
            Gt.idx[o] = G.idx[e];
            Gt.val[o] = G.val[e];
        }
        if (G.ptr[r + 1] - G.ptr[r] == 1) {
            Gt.idx[o] = G.ncols + bpre[r];
            Gt.val[o] = -G.val[G.ptr[r]];
        }
    }
    return Gt;
}

// -------------------------------------------------------------------------------------------
// Nodal graph (Section 4.1, reading of Alg. 2's "classical C/F splitting"): between gradient
// modes (original columns of G) a Ruge-Stueben strong connection of A_G = G^T A G in either
// direction, -a_ij >= theta max_{k != i}(-a_ik); any two columns of G~ sharing a row (edge).
// -------------------------------------------------------------------------------------------
// CSR from (row, col) pairs: rows sorted and deduplicated
static HostCSR csr_from_pairs(int n, const std::vector<std::vector<std::pair<int32_t, int32_t>>>& parts,
                              int nthreads) {
    HostCSR M;
    M.nrows = M.ncols = n;
    M.ptr.assign(n + 1, 0);
    for (const auto& p : parts)
        for (const auto& e : p) M.ptr[e.first + 1]++;
    for (int r = 0; r < n; ++r) M.ptr[r + 1] += M.ptr[r];
    M.idx.resize(M.ptr[n]);
    std::vector<int32_t> cur(M.ptr.begin(), M.ptr.end() - 1);
    for (const auto& p : parts)
        for (const auto& e : p) M.idx[cur[e.first]++] = e.second;
    // sort + unique each row, then compact
    std::vector<int32_t> newlen(n);
#pragma omp parallel for schedule(dynamic, 2048) num_threads(nthreads)
    for (int r = 0; r < n; ++r) {
        auto b = M.idx.begin() + M.ptr[r], e = M.idx.begin() + M.ptr[r + 1];
        std::sort(b, e);
        newlen[r] = (int32_t)(std::unique(b, e) - b);
    }
    std::vector<int32_t> ptr(n + 1, 0);
    for (int r = 0; r < n; ++r) ptr[r + 1] = ptr[r] + newlen[r];
    std::vector<int32_t> idx(ptr[n]);
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int r = 0; r < n; ++r) std::copy(M.idx.begin() + M.ptr[r], M.idx.begin() + M.ptr[r] + newlen[r], idx.begin() + ptr[r]);
    M.ptr.swap(ptr);
    M.idx.swap(idx);
    return M;
}

// -------------------------------------------------------------------------------------------
// Nodal graph (Section 4.1, reading of Alg. 2's "classical C/F splitting"): between gradient
// modes (original columns of G) a Ruge-Stueben strong connection of A_G = G^T A G in either
// direction, -a_ij >= theta max_{k != i}(-a_ik); any two columns of G~ sharing a row (edge).
// -------------------------------------------------------------------------------------------
static HostCSR nodal_graph(const HostCSR& A, const HostCSR& G, const HostCSR& Gt, const HostCSR& GtT,
                           double theta, int nthreads, HostCSR& Minc) {
    const int m = G.ncols, nn = Gt.ncols, ne = A.nrows;
    (void)GtT;
    HostCSR GT = transpose_pattern(G, true, nthreads);   // CSC of G: rows of column i with values
    // incidence pairs: columns sharing a row of G~
    std::vector<std::vector<std::pair<int32_t, int32_t>>> incp(nthreads);
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int r = 0; r < Gt.nrows; ++r) {
        if (Gt.ptr[r + 1] - Gt.ptr[r] != 2) continue;
        const int32_t a = Gt.idx[Gt.ptr[r]], b = Gt.idx[Gt.ptr[r] + 1];
        auto& v = incp[thread_id()];
        v.push_back({a, b});
        v.push_back({b, a});
    }
    Minc = csr_from_pairs(nn, incp, nthreads);
    PhaseClock nclk;
    // S: row i holds the strong connections of gradient mode i in A_G = G^T A G (sorted).  Each
    // thread takes one contiguous range of rows, so the threads' outputs concatenate into CSR.
    HostCSR S;
    S.nrows = S.ncols = nn;
    S.ptr.assign(nn + 1, 0);
    std::vector<std::vector<int32_t>> sidx(nthreads);
    std::vector<int32_t> slen(nn, 0);
#pragma omp parallel num_threads(nthreads)
    {
        const int tid = thread_id(), nt = omp_threads();
        const int i0 = (int)((int64_t)m * tid / nt), i1 = (int)((int64_t)m * (tid + 1) / nt);
        std::vector<int32_t> wm(ne, -1), am(m, -1), tf, tj;
        std::vector<double> wv(ne, 0.0), av(m, 0.0);
        auto& out = sidx[tid];
        for (int i = i0; i < i1; ++i) {
            tf.clear();
            tj.clear();
            // w = A g_i over the edges of node i (A symmetric: column e of A is row e)
            for (int32_t t = GT.ptr[i]; t < GT.ptr[i + 1]; ++t) {
                const int32_t e = GT.idx[t];
                const double ge = GT.val[t];
                for (int32_t q = A.ptr[e]; q < A.ptr[e + 1]; ++q) {
                    const int32_t f = A.idx[q];
                    if (wm[f] != i) { wm[f] = i; wv[f] = 0.0; tf.push_back(f); }
                    wv[f] += ge * A.val[q];
                }
            }
            // row i of G^T A G
            for (int32_t f : tf)
                for (int32_t u = G.ptr[f]; u < G.ptr[f + 1]; ++u) {
                    const int32_t j = G.idx[u];
                    if (am[j] != i) { am[j] = i; av[j] = 0.0; tj.push_back(j); }
                    av[j] += G.val[u] * wv[f];
                }
            double rowmax = -INFINITY;
            for (int32_t j : tj)
                if (j != i) rowmax = std::max(rowmax, -av[j]);
            const size_t b = out.size();
            if (rowmax > 0.0)
                for (int32_t j : tj)
                    if (j != i && -av[j] >= theta * rowmax) out.push_back(j);
            std::sort(out.begin() + b, out.end());
            slen[i] = (int32_t)(out.size() - b);
        }
    }
    for (int i = 0; i < nn; ++i) S.ptr[i + 1] = S.ptr[i] + slen[i];
    for (const auto& v : sidx) S.idx.insert(S.idx.end(), v.begin(), v.end());
    nclk.mark("  strong connections");
    HostCSR ST = transpose_pattern(S, false, nthreads);
    // N = S + S^T + incidence, row by row as sorted unions
    HostCSR N;
    N.nrows = N.ncols = nn;
    N.ptr.assign(nn + 1, 0);
    auto merged = [&](int r, int32_t* dst) {
        const HostCSR* M3[3] = {&S, &ST, &Minc};
        int32_t pos[3], end[3];
        for (int k = 0; k < 3; ++k) {
            pos[k] = M3[k]->ptr[r];
            end[k] = M3[k]->ptr[r + 1];
        }
        int cnt = 0;
        int32_t last = -1;
        for (;;) {
            int32_t best = INT32_MAX;
            for (int k = 0; k < 3; ++k)
                if (pos[k] < end[k]) best = std::min(best, M3[k]->idx[pos[k]]);
            if (best == INT32_MAX) break;
            for (int k = 0; k < 3; ++k)
                if (pos[k] < end[k] && M3[k]->idx[pos[k]] == best) pos[k]++;
            if (best != last) {
                if (dst) dst[cnt] = best;
                cnt++;
                last = best;
            }
        }
        return cnt;
    };
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int r = 0; r < nn; ++r) N.ptr[r + 1] = merged(r, nullptr);
    for (int r = 0; r < nn; ++r) N.ptr[r + 1] += N.ptr[r];
    N.idx.resize(N.ptr[nn]);
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int r = 0; r < nn; ++r) merged(r, N.idx.data() + N.ptr[r]);
    nclk.mark("  transpose + union");
    return N;
}

// -------------------------------------------------------------------------------------------
// Alg. 2: C starts as the artificial boundary columns, their neighbours start as F, then the
// Ruge-Stueben first pass (measure |N & U| + 2 |N & F|, largest first, ties to the smallest
// index) splits the remaining nodes; nodes without neighbours are F.
// -------------------------------------------------------------------------------------------
enum : int8_t { ST_U = 0, ST_C = 1, ST_F = 2 };

// Nodes bucketed by their measure; a bucket is a two-level bitset over the node indices, so that
// the node of largest measure and, among those, of smallest index is found by scanning a few
// summary words, and a measure increment moves a node between buckets in O(1).
class BucketQueue {
   public:
    explicit BucketQueue(int n) : n_(n), w_((n + 63) / 64), s_((w_ + 63) / 64) {}
    void insert(int64_t b, int i) {
        ensure(b);
        auto& lo = lo_[b];
        if (!lo[i >> 6]) hi_[b][i >> 12] |= 1ull << ((i >> 6) & 63);
        lo[i >> 6] |= 1ull << (i & 63);
        count_[b]++;
        if (b > top_) top_ = b;
    }
    void erase(int64_t b, int i) {
        auto& lo = lo_[b];
        lo[i >> 6] &= ~(1ull << (i & 63));
        if (!lo[i >> 6]) hi_[b][i >> 12] &= ~(1ull << ((i >> 6) & 63));
        count_[b]--;
    }
    // node of largest measure, smallest index among equals; -1 when empty
    int top(int64_t* bucket) {
        while (top_ >= 0 && count_[top_] == 0) --top_;
        if (top_ < 0) return -1;
        const auto& hi = hi_[top_];
        const auto& lo = lo_[top_];
        for (int s = 0; s < s_; ++s)
            if (hi[s]) {
                const int w = s * 64 + __builtin_ctzll(hi[s]);
                *bucket = top_;
                return w * 64 + __builtin_ctzll(lo[w]);
            }
        return -1;
    }

   private:
    void ensure(int64_t b) {
        while ((int64_t)lo_.size() <= b) {
            lo_.emplace_back(w_, 0ull);
            hi_.emplace_back(s_, 0ull);
            count_.push_back(0);
        }
    }
    int n_, w_, s_;
    int64_t top_ = -1;
    std::vector<std::vector<uint64_t>> lo_, hi_;
    std::vector<int64_t> count_;
};

static void nodal_cf(const HostCSR& N, int m, std::vector<int8_t>& st) {
    const int nn = N.nrows;
    st.assign(nn, ST_U);
    for (int b = m; b < nn; ++b) st[b] = ST_C;
    for (int b = m; b < nn; ++b)
        for (int32_t t = N.ptr[b]; t < N.ptr[b + 1]; ++t)
            if (st[N.idx[t]] == ST_U) st[N.idx[t]] = ST_F;
    for (int i = 0; i < nn; ++i)
        if (st[i] == ST_U && N.ptr[i + 1] == N.ptr[i]) st[i] = ST_F;
    std::vector<int64_t> lam(nn, 0);
    BucketQueue q(nn);
    for (int i = 0; i < nn; ++i) {
        if (st[i] != ST_U) continue;
        int64_t l = 0;
        for (int32_t t = N.ptr[i]; t < N.ptr[i + 1]; ++t) {
            int8_t s = st[N.idx[t]];
            l += (s == ST_U) ? 1 : (s == ST_F ? 2 : 0);
        }
        lam[i] = l;
        q.insert(l, i);
    }
    std::vector<int32_t> newf;
    int64_t b = 0;
    for (int i = q.top(&b); i >= 0; i = q.top(&b)) {
        q.erase(b, i);
        st[i] = ST_C;
        newf.clear();
        for (int32_t t = N.ptr[i]; t < N.ptr[i + 1]; ++t) {
            const int32_t j = N.idx[t];
            if (st[j] == ST_U) {
                st[j] = ST_F;
                q.erase(lam[j], j);
                newf.push_back(j);
            }
        }
        for (int32_t j : newf)
            for (int32_t t = N.ptr[j]; t < N.ptr[j + 1]; ++t) {
                const int32_t l = N.idx[t];
                if (st[l] == ST_U) {
                    q.erase(lam[l], l);
                    q.insert(++lam[l], l);
                }
            }
    }
}

// -------------------------------------------------------------------------------------------
// Alg. 3, enumerated around the middle node: every pair (a, b) of coarse columns (C = c_G u B)
// in M(k), a < b, not both artificial, not neighbours, has k as a candidate.  Sorting the triples
// (a, b, k) visits the pairs in the order of the pair loop over C x C, and the first candidate
// k not yet used is taken (R: smallest middle node), which reproduces Alg. 3 exactly.
// -------------------------------------------------------------------------------------------
static void match(const HostCSR& Gt, const HostCSR& GtT, const HostCSR& N, const HostCSR& M,
                  const std::vector<int8_t>& st, int m, std::vector<CoarseEdge>& out) {
    const int nn = N.nrows;
    struct Tri { int32_t a, b, k; };
    std::vector<Tri> tri;
    std::vector<int32_t> cand;
    for (int k = 0; k < nn; ++k) {
        cand.clear();
        for (int32_t t = M.ptr[k]; t < M.ptr[k + 1]; ++t)
            if (st[M.idx[t]] == ST_C) cand.push_back(M.idx[t]);
        for (size_t x = 0; x < cand.size(); ++x)
            for (size_t y = x + 1; y < cand.size(); ++y) {
                int32_t a = cand[x], b = cand[y];
                if (a >= m && b >= m) continue;           // (i, j) both artificial
                if (has(N, a, b)) continue;               // neighbours: not at distance two
                if (!has(N, a, k) || !has(N, b, k)) continue;
                tri.push_back({a, b, k});
            }
    }
    std::sort(tri.begin(), tri.end(), [](const Tri& x, const Tri& y) {
        if (x.a != y.a) return x.a < y.a;
        if (x.b != y.b) return x.b < y.b;
        return x.k < y.k;
    });
    std::vector<char> used(nn, 0);
    auto edge_between = [&](int32_t u, int32_t v) -> int32_t {   // smallest row of G~ holding u and v
        for (int32_t t = GtT.ptr[v]; t < GtT.ptr[v + 1]; ++t) {
            int32_t r = GtT.idx[t];
            if (Gt.ptr[r + 1] - Gt.ptr[r] == 2 && (Gt.idx[Gt.ptr[r]] == u || Gt.idx[Gt.ptr[r] + 1] == u)) return r;
        }
        return -1;
    };
    auto value_at = [&](int32_t r, int32_t c) -> int32_t {
        for (int32_t u = Gt.ptr[r]; u < Gt.ptr[r + 1]; ++u)
            if (Gt.idx[u] == c) return (int32_t)Gt.val[u];
        return 0;
    };
    size_t p = 0;
    while (p < tri.size()) {
        size_t q = p;
        while (q < tri.size() && tri[q].a == tri[p].a && tri[q].b == tri[p].b) ++q;
        for (size_t s = p; s < q; ++s) {
            int32_t k = tri[s].k;
            if (used[k]) continue;
            int32_t i = tri[s].a, j = tri[s].b;
            int32_t d1 = edge_between(i, k), d2 = edge_between(j, k);
            used[k] = 1;
            out.push_back({d1, value_at(d1, k), d2, -value_at(d2, k), i, k, j});
            break;
        }
        p = q;
    }
}

static std::string finish_coarsening(const HostCSR& A, const HostCSR& G, const Params& prm, Coarsening& out,
                                     int nthreads, PhaseClock& clk);

std::string coarsen_level(const HostCSR& A, const HostCSR& G, const Params& prm, Coarsening& out,
                          int nthreads) {
    PhaseClock clk;
    int nB = 0;
    HostCSR Gt = augment(G, nB, nthreads);
    HostCSR GtT = transpose_pattern(Gt, false, nthreads);
    clk.mark("augment");
    HostCSR Minc;
    HostCSR N = nodal_graph(A, G, Gt, GtT, prm.theta, nthreads, Minc);
    clk.mark("nodal graph");
    out.m = G.ncols;
    out.nB = nB;
    nodal_cf(N, G.ncols, out.state);
    clk.mark("nodal C/F");
    out.edges.clear();
    match(Gt, GtT, N, Minc, out.state, G.ncols, out.edges);
    clk.mark("matching");
    if (out.edges.empty()) return "";
    for (const auto& e : out.edges)
        if (e.d1 < 0 || e.d2 < 0) return "internal: matching found no edge for a path";
    out.geo_ptr.clear();
    out.geo_idx.clear();
    out.geo_val.clear();
    return finish_coarsening(A, G, prm, out, nthreads, clk);
}

// -------------------------------------------------------------------------------------------
// Section 3's refinement-based coarse variables on the structured hex mesh of the unit cube with
// mesh_n intervals per side (interior edges numbered x, y, z, each lexicographic by start node,
// +axis; interior nodes lexicographic).  Every interior edge of the coarse (mesh_n/2)^3 mesh, in
// the coarse mesh's own numbering, pairs its two fine halves with signs (+1, +1): the orthogonal
// complement of the middle node's gradient column, both halves oriented like the coarse edge.
// With `geometric`, the interior support of a column is the 16 fine edges parallel to it one fine
// step across (the support of the geometric Nedelec interpolation), with the hat-product weights
// 1/2 (one transverse step) and 1/4 (two), in the scaling whose rows on the halves are R^T.
// -------------------------------------------------------------------------------------------
namespace {
struct HexIds {
    int n, m;
    int64_t nx;
    explicit HexIds(int nn) : n(nn), m(nn - 1), nx((int64_t)nn * (nn - 1) * (nn - 1)) {}
    int32_t edge(int d, int i, int j, int k) const {
        if (d == 0) return (i >= 0 && i < n && j >= 1 && j <= m && k >= 1 && k <= m)
                               ? (int32_t)(i + (int64_t)n * ((j - 1) + (int64_t)m * (k - 1))) : -1;
        if (d == 1) return (i >= 1 && i <= m && j >= 0 && j < n && k >= 1 && k <= m)
                               ? (int32_t)(nx + (i - 1) + (int64_t)m * (j + (int64_t)n * (k - 1))) : -1;
        return (i >= 1 && i <= m && j >= 1 && j <= m && k >= 0 && k < n)
                   ? (int32_t)(2 * nx + (i - 1) + (int64_t)m * ((j - 1) + (int64_t)m * k)) : -1;
    }
    int32_t node(int i, int j, int k) const {
        return (i >= 1 && i <= m && j >= 1 && j <= m && k >= 1 && k <= m)
                   ? (int32_t)((i - 1) + (int64_t)m * ((j - 1) + (int64_t)m * (k - 1))) : -1;
    }
    int64_t nedges() const { return 3 * nx; }
};
}  // namespace

std::string coarsen_level_refinement(const HostCSR& A, const HostCSR& G, int mesh_n, bool geometric,
                                     const Params& prm, Coarsening& out, int nthreads) {
    PhaseClock clk;
    if (mesh_n < 4 || mesh_n % 2) return "refinement coarsening needs an even mesh size of at least 4";
    const HexIds fine(mesh_n), coarse(mesh_n / 2);
    if (A.nrows != fine.nedges() || G.nrows != A.nrows || G.ncols != (int64_t)fine.m * fine.m * fine.m)
        return "A and G do not match a hex mesh of " + std::to_string(mesh_n) + " intervals per side";
    const int N = mesh_n / 2;
    const int nc = (int)coarse.nedges();
    out.edges.assign(nc, CoarseEdge{-1, 0, -1, 0, -1, -1, -1});
    out.m = G.ncols;
    out.nB = 0;
    out.state.assign(G.ncols, 2);
    const int step[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int d = 0; d < 3; ++d)
        for (int K = 0; K <= N; ++K)
            for (int J = 0; J <= N; ++J)
                for (int I = 0; I <= N; ++I) {
                    const int32_t c = coarse.edge(d, I, J, K);
                    if (c < 0) continue;
                    const int x = 2 * I, y = 2 * J, z = 2 * K, a = step[d][0], b = step[d][1], e = step[d][2];
                    CoarseEdge& ce = out.edges[c];
                    ce.d1 = fine.edge(d, x, y, z);
                    ce.d2 = fine.edge(d, x + a, y + b, z + e);
                    ce.s1 = ce.s2 = 1;
                    ce.i = fine.node(x, y, z);
                    ce.k = fine.node(x + a, y + b, z + e);
                    ce.j = fine.node(x + 2 * a, y + 2 * b, z + 2 * e);
                    if (ce.d1 < 0 || ce.d2 < 0 || ce.k < 0) return "internal: a coarse edge's half is not interior";
                    if (ce.i >= 0) out.state[ce.i] = 1;
                    if (ce.j >= 0) out.state[ce.j] = 1;
                }
    clk.mark("refinement pairs");
    out.geo_ptr.clear();
    out.geo_idx.clear();
    out.geo_val.clear();
    if (!geometric) return finish_coarsening(A, G, prm, out, nthreads, clk);
    // geometric interpolation: the supports and weights of Sec. 5's comparison interpolation
    out.geo_ptr.assign(nc + 1, 0);
    out.geo_idx.clear();
    out.geo_val.clear();
    for (int d = 0; d < 3; ++d)
        for (int K = 0; K <= N; ++K)
            for (int J = 0; J <= N; ++J)
                for (int I = 0; I <= N; ++I) {
                    const int32_t c = coarse.edge(d, I, J, K);
                    if (c < 0) continue;
                    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
                    std::vector<std::pair<int32_t, double>> col;
                    for (int half = 0; half < 2; ++half)
                        for (int o1 = -1; o1 <= 1; ++o1)
                            for (int o2 = -1; o2 <= 1; ++o2) {
                                if (o1 == 0 && o2 == 0) continue;   // the halves: R^T
                                int q[3] = {2 * I + half * step[d][0], 2 * J + half * step[d][1],
                                            2 * K + half * step[d][2]};
                                q[t1] += o1;
                                q[t2] += o2;
                                const int32_t f = fine.edge(d, q[0], q[1], q[2]);
                                if (f >= 0) col.push_back({f, (o1 ? 0.5 : 1.0) * (o2 ? 0.5 : 1.0)});
                            }
                    std::sort(col.begin(), col.end());
                    for (const auto& pv : col) {
                        out.geo_idx.push_back(pv.first);
                        out.geo_val.push_back(pv.second);
                    }
                    out.geo_ptr[c + 1] = (int32_t)col.size();
                }
    for (int c = 0; c < nc; ++c) out.geo_ptr[c + 1] += out.geo_ptr[c];
    // the columns were appended in the loop order, which is the coarse numbering's order
    clk.mark("geometric interpolation");
    return finish_coarsening(A, G, prm, out, nthreads, clk);
}

static std::string finish_coarsening(const HostCSR& A, const HostCSR& G, const Params& prm, Coarsening& out,
                                     int nthreads, PhaseClock& clk) {
    const int n = A.nrows;
    const int nc = (int)out.edges.size();
    // Eq. Gc: rows e_j - e_i over the ends that are columns of G (an artificial or eliminated
    // end contributes nothing); keep the nonzero columns
    std::vector<char> keep(G.ncols, 0);
    for (const auto& e : out.edges) {
        if (e.i >= 0 && e.i < G.ncols) keep[e.i] = 1;
        if (e.j >= 0 && e.j < G.ncols) keep[e.j] = 1;
    }
    std::vector<int32_t> newid(G.ncols, -1);
    out.coarse_nodes.clear();
    for (int v = 0; v < G.ncols; ++v)
        if (keep[v]) {
            newid[v] = (int32_t)out.coarse_nodes.size();
            out.coarse_nodes.push_back(v);
        }
    HostCSR& Gc = out.Gc;
    Gc.nrows = nc;
    Gc.ncols = (int)out.coarse_nodes.size();
    Gc.ptr.assign(nc + 1, 0);
    Gc.idx.clear();
    Gc.val.clear();
    for (int c = 0; c < nc; ++c) {
        const auto& e = out.edges[c];
        // new ids keep the order of the fine columns, so the row stays sorted when i < j
        const bool hi = e.i >= 0 && e.i < G.ncols, hj = e.j >= 0 && e.j < G.ncols;
        if (hi && hj && e.j < e.i) return "internal: a coarse edge's ends are out of order";
        if (hi) {
            Gc.idx.push_back(newid[e.i]);
            Gc.val.push_back(-1.0);
        }
        if (hj) {
            Gc.idx.push_back(newid[e.j]);
            Gc.val.push_back(1.0);
        }
        Gc.ptr[c + 1] = (int32_t)Gc.idx.size();
    }

    if (!out.geo_ptr.empty()) {
        // the geometric interpolation's supports stand in for the patches (their values are set,
        // not solved for)
        out.patch_ptr = out.geo_ptr;
        out.patch_idx = out.geo_idx;
    } else {
        // ---- Eq. sparseP patches: components of graph(A_II) if small enough, else rings ----------
        std::vector<char> ext(n, 0);
        for (const auto& e : out.edges) ext[e.d1] = ext[e.d2] = 1;
        // connected components of graph(A_II) by a concurrent union-find: a root is only ever linked
        // below a smaller root (compare-and-swap), so every component ends with its smallest member as
        // root whatever the order of the unions; finds halve paths with relaxed stores, which keep
        // every node's parent an ancestor
        std::vector<int32_t> parent(n);
        std::iota(parent.begin(), parent.end(), 0);
        int32_t* par = parent.data();
        auto find = [par](int32_t x) {
            for (;;) {
                const int32_t p = __atomic_load_n(&par[x], __ATOMIC_RELAXED);
                if (p == x) return x;
                const int32_t gp = __atomic_load_n(&par[p], __ATOMIC_RELAXED);
                if (gp != p) __atomic_store_n(&par[x], gp, __ATOMIC_RELAXED);
                x = gp;
            }
        };
    #pragma omp parallel for schedule(dynamic, 4096) num_threads(nthreads)
        for (int r = 0; r < n; ++r) {
            if (ext[r]) continue;
            for (int32_t t = A.ptr[r]; t < A.ptr[r + 1]; ++t) {
                const int32_t c = A.idx[t];
                if (c <= r || ext[c]) continue;
                int32_t x = r, y = c;
                for (;;) {
                    x = find(x);
                    y = find(y);
                    if (x == y) break;
                    if (x < y) std::swap(x, y);   // link the larger root below the smaller one
                    int32_t expect = x;
                    if (__atomic_compare_exchange_n(&par[x], &expect, y, false, __ATOMIC_ACQ_REL, __ATOMIC_RELAXED)) break;
                }
            }
        }
        std::vector<int32_t> comp(n, -1), csize;
        {
            std::vector<int32_t> label(n, -1);
            for (int r = 0; r < n; ++r)
                if (!ext[r]) {
                    int32_t root = find(r);
                    if (label[root] < 0) { label[root] = (int32_t)csize.size(); csize.push_back(0); }
                    comp[r] = label[root];
                    csize[comp[r]]++;
                }
        }
        std::vector<int32_t> cptr(csize.size() + 1, 0), cmem(n);
        for (size_t c = 0; c < csize.size(); ++c) cptr[c + 1] = cptr[c] + csize[c];
        {
            std::vector<int32_t> cur(cptr.begin(), cptr.end() - 1);
            for (int r = 0; r < n; ++r)
                if (comp[r] >= 0) cmem[cur[comp[r]]++] = r;   // ascending within a component
        }
        clk.mark("G_c + components");
        // each thread keeps its scratch lists across coarse edges and appends the patches it builds
        // to its own flat buffer; a patch is found through (thread, offset, length)
        std::vector<std::vector<int32_t>> pbuf(nthreads);
        std::vector<int32_t> pthread(nc), poff(nc), plen(nc);
    #pragma omp parallel num_threads(nthreads)
        {
            const int tid = thread_id();
            auto& buf = pbuf[tid];
            std::vector<int32_t> seeds, comps, order, level, seen, nxt, merged;
    #pragma omp for schedule(dynamic, 64)
            for (int c = 0; c < nc; ++c) {
                const auto& e = out.edges[c];
                seeds.clear();
                for (int32_t d : {e.d1, e.d2})
                    for (int32_t t = A.ptr[d]; t < A.ptr[d + 1]; ++t)
                        if (!ext[A.idx[t]]) seeds.push_back(A.idx[t]);
                std::sort(seeds.begin(), seeds.end());
                seeds.erase(std::unique(seeds.begin(), seeds.end()), seeds.end());
                comps.clear();
                for (int32_t sd : seeds) comps.push_back(comp[sd]);
                std::sort(comps.begin(), comps.end());
                comps.erase(std::unique(comps.begin(), comps.end()), comps.end());
                int64_t tot = 0;
                for (int32_t q : comps) tot += csize[q];
                const size_t b = buf.size();
                if (tot <= prm.p_max) {
                    for (int32_t q : comps) buf.insert(buf.end(), cmem.begin() + cptr[q], cmem.begin() + cptr[q + 1]);
                } else {
                    order = seeds;
                    level = seeds;
                    seen = seeds;   // sorted
                    for (int r = 1; r < prm.ring && (int)order.size() < prm.p_max; ++r) {
                        nxt.clear();
                        for (int32_t d : level)
                            for (int32_t t = A.ptr[d]; t < A.ptr[d + 1]; ++t) {
                                int32_t x = A.idx[t];
                                if (!ext[x] && !std::binary_search(seen.begin(), seen.end(), x)) nxt.push_back(x);
                            }
                        std::sort(nxt.begin(), nxt.end());
                        nxt.erase(std::unique(nxt.begin(), nxt.end()), nxt.end());
                        order.insert(order.end(), nxt.begin(), nxt.end());
                        merged.clear();
                        std::merge(seen.begin(), seen.end(), nxt.begin(), nxt.end(), std::back_inserter(merged));
                        seen.swap(merged);
                        level.swap(nxt);
                    }
                    if ((int)order.size() > prm.p_max) order.resize(prm.p_max);
                    buf.insert(buf.end(), order.begin(), order.end());
                }
                std::sort(buf.begin() + (std::ptrdiff_t)b, buf.end());
                pthread[c] = tid;
                poff[c] = (int32_t)b;
                plen[c] = (int32_t)(buf.size() - b);
            }
        }
        out.patch_ptr.assign(nc + 1, 0);
        for (int c = 0; c < nc; ++c) out.patch_ptr[c + 1] = out.patch_ptr[c] + plen[c];
        out.patch_idx.resize(out.patch_ptr[nc]);
    #pragma omp parallel for schedule(static) num_threads(nthreads)
        for (int c = 0; c < nc; ++c) {
            const int32_t* src = pbuf[pthread[c]].data() + poff[c];
            std::copy(src, src + plen[c], out.patch_idx.begin() + out.patch_ptr[c]);
        }
    }
    clk.mark("patches");
    // ---- patterns of P^T (row c: the patch and the two exterior DoFs, ascending) and of P (its
    // transpose), with the positions of every computed entry in both -------------------------
    HostCSR& PT = out.PT;
    PT.nrows = nc;
    PT.ncols = n;
    PT.ptr.assign(nc + 1, 0);
    for (int c = 0; c < nc; ++c) PT.ptr[c + 1] = PT.ptr[c] + 2 + (out.patch_ptr[c + 1] - out.patch_ptr[c]);
    PT.idx.assign(PT.ptr[nc], 0);
    PT.val.assign(PT.ptr[nc], 0.0);
    out.patch_pos_PT.assign(out.patch_idx.size(), 0);
    out.ext_pos_PT.assign(2 * (size_t)nc, 0);
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
    for (int c = 0; c < nc; ++c) {
        const auto& e = out.edges[c];
        int32_t pos = PT.ptr[c];
        int32_t a = out.patch_ptr[c], aend = out.patch_ptr[c + 1];
        int32_t ex[2] = {std::min(e.d1, e.d2), std::max(e.d1, e.d2)};
        double exv[2] = {(double)(e.d1 < e.d2 ? e.s1 : e.s2), (double)(e.d1 < e.d2 ? e.s2 : e.s1)};
        int xi = 0;
        while (a < aend || xi < 2) {
            if (xi < 2 && (a >= aend || ex[xi] < out.patch_idx[a])) {
                PT.idx[pos] = ex[xi];
                PT.val[pos] = exv[xi];
                out.ext_pos_PT[2 * c + ((ex[xi] == e.d1) ? 0 : 1)] = pos;
                ++xi;
            } else {
                PT.idx[pos] = out.patch_idx[a];
                out.patch_pos_PT[a] = pos;
                ++a;
            }
            ++pos;
        }
    }
    clk.mark("P^T pattern");
    HostCSR& P = out.P;
    P.nrows = n;
    P.ncols = nc;
    P.ptr.assign(n + 1, 0);
    const int64_t nzp = PT.ptr[nc];
    std::vector<int32_t> fromPT(nzp);   // P position -> P^T position
    std::vector<int32_t> toP(nzp);      // P^T position -> P position
    {
        // counting sort of the P^T entries by row of P; each thread scatters one contiguous range
        // of coarse edges, and per-thread offsets keep every row in ascending column order
        const int nt = std::max(1, nthreads);
        std::vector<std::vector<int32_t>> cnt(nt);
#pragma omp parallel num_threads(nt)
        {
            const int tid = thread_id(), ntr = omp_threads();
            const int c0 = (int)((int64_t)nc * tid / ntr), c1 = (int)((int64_t)nc * (tid + 1) / ntr);
            auto& v = cnt[tid];
            v.assign(n, 0);
            for (int32_t q = PT.ptr[c0]; q < PT.ptr[c1]; ++q) v[PT.idx[q]]++;
#pragma omp barrier
#pragma omp for schedule(static)
            for (int r = 0; r < n; ++r) {
                int32_t s = 0;
                for (int t = 0; t < ntr; ++t) s += cnt[t][r];
                P.ptr[r + 1] = s;
            }
#pragma omp single
            for (int r = 0; r < n; ++r) P.ptr[r + 1] += P.ptr[r];
#pragma omp for schedule(static)
            for (int r = 0; r < n; ++r) {
                int32_t off = P.ptr[r];
                for (int t = 0; t < ntr; ++t) {
                    const int32_t k = cnt[t][r];
                    cnt[t][r] = off;
                    off += k;
                }
            }
            for (int c = c0; c < c1; ++c)
                for (int32_t q = PT.ptr[c]; q < PT.ptr[c + 1]; ++q) {
                    const int32_t pp = v[PT.idx[q]]++;
                    fromPT[pp] = q;
                    toP[q] = pp;
                }
        }
    }
    P.idx.resize(nzp);
    P.val.resize(nzp);
    int32_t* cidx = P.idx.data();
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int c = 0; c < nc; ++c)
        for (int32_t q = PT.ptr[c]; q < PT.ptr[c + 1]; ++q) {
            cidx[toP[q]] = c;
            P.val[toP[q]] = PT.val[q];
        }
    out.patch_pos_P.assign(out.patch_idx.size(), 0);
    out.ext_pos_P.assign(2 * (size_t)nc, 0);
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t t = 0; t < (int64_t)out.patch_idx.size(); ++t) out.patch_pos_P[t] = toP[out.patch_pos_PT[t]];
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t t = 0; t < 2 * (int64_t)nc; ++t) out.ext_pos_P[t] = toP[out.ext_pos_PT[t]];

    // ---- symbolic Galerkin patterns ----------------------------------------------------------
    clk.mark("P pattern");
    if (prm.symbolic_galerkin) {
        out.AP = symbolic_rows(A, P, nthreads);
        clk.mark("symbolic AP");
        out.Ac = symbolic_rows(PT, out.AP, nthreads);
        clk.mark("symbolic PtAP");
    }
    return "";
}

// -------------------------------------------------------------------------------------------
// OSS-l1 smoother structure: node stars of G, greedy colouring of "an entry of A couples two
// stars", and the warp slot layout (stars of one colour packed into 32-lane groups).
// -------------------------------------------------------------------------------------------
std::string build_stars(const HostCSR& A, const HostCSR& G, StarLayout& L) {
    PhaseClock clk;
    HostCSR GT = transpose_pattern(G, false);
    const int ns = G.ncols;
    L.nstars = ns;
    L.star_ptr = GT.ptr;
    L.star_idx = GT.idx;
    L.max_block = 0;
    for (int j = 0; j < ns; ++j) L.max_block = std::max(L.max_block, GT.ptr[j + 1] - GT.ptr[j]);
    if (L.max_block > 32) return "smoother star of " + std::to_string(L.max_block) + " DoFs exceeds 32";
    // conflict lists in parallel (star j ~ j' when an entry of A couples them), then the greedy
    // pass in ascending j, which is inherently sequential.  Each thread takes contiguous blocks of
    // stars and appends their (lower) conflict lists to its own flat buffer; a star's list is
    // found through (thread, offset, length), so no per-star allocation is made.
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = std::max(1, std::min(omp_get_max_threads(), 32));
#endif
    std::vector<std::vector<int32_t>> stamps(nthreads), lists(nthreads);
    std::vector<int32_t> lthread(ns), loff(ns), llen(ns);
#pragma omp parallel num_threads(nthreads)
    {
        const int tid = thread_id();
        auto& stamp = stamps[tid];
        stamp.assign(ns, -1);
        auto& buf = lists[tid];
#pragma omp for schedule(dynamic, 512)
        for (int j = 0; j < ns; ++j) {
            const size_t b = buf.size();
            for (int32_t t = GT.ptr[j]; t < GT.ptr[j + 1]; ++t) {
                int32_t e = GT.idx[t];
                for (int32_t q = A.ptr[e]; q < A.ptr[e + 1]; ++q) {
                    int32_t f = A.idx[q];
                    for (int32_t u = G.ptr[f]; u < G.ptr[f + 1]; ++u) {
                        int32_t jj = G.idx[u];
                        if (jj < j && stamp[jj] != j) { stamp[jj] = j; buf.push_back(jj); }
                    }
                }
            }
            lthread[j] = tid;
            loff[j] = (int32_t)b;
            llen[j] = (int32_t)(buf.size() - b);
        }
    }
    L.colour.assign(ns, -1);
    std::vector<int32_t> mark;   // mark[c] == j: colour c is taken by a neighbour of star j
    int ncol = 0;
    for (int j = 0; j < ns; ++j) {
        if ((int)mark.size() < ncol + 1) mark.resize(ncol + 1, -1);
        const int32_t* nb = lists[lthread[j]].data() + loff[j];
        for (int32_t q = 0; q < llen[j]; ++q) mark[L.colour[nb[q]]] = j;
        int c = 0;
        while (c < ncol && mark[c] == j) ++c;
        L.colour[j] = c;
        ncol = std::max(ncol, c + 1);
    }
    L.ncolours = ncol;
    clk.mark("stars + colouring");
    return "";
}

// ---- Eq. commuting: nodal interpolation and the per-row data of the least-distance correction ----
std::string commuting_rows(const HostCSR& G, const Coarsening& cz, CommutingRows& out, int nthreads) {
    PhaseClock clk;
    const int n = G.nrows, m = G.ncols;
    const HostCSR& P = cz.P;
    const HostCSR& PT = cz.PT;
    const HostCSR& Gc = cz.Gc;
    const int nc = (int)cz.edges.size();
    const int ncn = Gc.ncols;
    if (P.nrows != n || PT.nrows != nc || Gc.nrows != nc || (int)G.val.size() != (int)G.nnz())
        return "internal: commuting rows need G with values and the patterns of P, P^T and G_c";
    std::vector<int32_t> col(m, -1);
    for (size_t q = 0; q < cz.coarse_nodes.size(); ++q) col[cz.coarse_nodes[q]] = (int32_t)q;
    typedef std::pair<int32_t, double> Entry;

    // P_n row by row (ascending coarse node): row v at rowp[v], len[v] entries; layer 0 in `pool`,
    // every later layer in its own per-thread buffers
    std::vector<int32_t> len(m, 0), layer(m, -1);
    std::vector<const Entry*> rowp(m, nullptr);
    std::vector<int64_t> off(m, 0);
    std::vector<Entry> pool;
    pool.reserve((size_t)m + 2 * cz.edges.size());
    for (int v = 0; v < m; ++v)
        if (col[v] >= 0) {
            layer[v] = 0;
            off[v] = (int64_t)pool.size();
            len[v] = 1;
            pool.emplace_back(col[v], 1.0);
        }
    for (const auto& e : cz.edges) {
        if (e.k < 0 || e.k >= m) continue;
        if (layer[e.k] == 0) return "internal: a middle node is a coarse node or the middle of two pairs";
        layer[e.k] = 0;
        Entry row[2];
        int nr = 0;
        for (int32_t end : {e.i, e.j})
            if (end >= 0 && end < m && col[end] >= 0) row[nr++] = Entry(col[end], 0.5);
        if (nr == 2 && row[0].first == row[1].first) {
            row[0].second = 1.0;
            nr = 1;
        }
        if (nr == 2 && row[1].first < row[0].first) std::swap(row[0], row[1]);
        off[e.k] = (int64_t)pool.size();
        len[e.k] = nr;
        for (int t = 0; t < nr; ++t) pool.push_back(row[t]);
    }
    for (int v = 0; v < m; ++v)
        if (layer[v] == 0) rowp[v] = pool.data() + off[v];
    HostCSR GT = transpose_pattern(G, false, nthreads);   // node -> its rows of G
    auto other_end = [&](int32_t row, int32_t v) -> int32_t {
        const int32_t a = G.ptr[row], b = G.ptr[row + 1];
        if (b - a != 2) return -1;   // a boundary edge: its other end is artificial (zero)
        return G.idx[a] == v ? G.idx[a + 1] : G.idx[a];
    };
    const int nth = std::max(1, nthreads);
    std::vector<std::vector<std::vector<Entry>>> layer_bufs;
    for (int d = 1;; ++d) {
        // layer d: the unassigned nodes next to layer d - 1, found by a scan in node order (each
        // thread a contiguous range, so the concatenation is ascending)
        std::vector<std::vector<int32_t>> found(nth);
#pragma omp parallel num_threads(nth)
        {
            const int tid = thread_id();
            const int64_t lo = (int64_t)m * tid / nth, hi = (int64_t)m * (tid + 1) / nth;
            for (int64_t u = lo; u < hi; ++u) {
                if (layer[u] >= 0) continue;
                for (int32_t q = GT.ptr[u]; q < GT.ptr[u + 1]; ++q) {
                    const int32_t w = other_end(GT.idx[q], (int32_t)u);
                    if (w >= 0 && layer[w] == d - 1) {
                        found[tid].push_back((int32_t)u);
                        break;
                    }
                }
            }
        }
        std::vector<int32_t> next;
        for (const auto& f : found) next.insert(next.end(), f.begin(), f.end());
        if (next.empty()) break;
        for (int32_t w : next) layer[w] = d;
        // each new row: the mean over the previous layer's neighbours and the boundary edges
        layer_bufs.emplace_back(nth);
        auto& tbuf = layer_bufs.back();
        std::vector<int32_t> bthread(next.size());
        std::vector<int64_t> boff(next.size());
#pragma omp parallel num_threads(nth)
        {
            const int tid = thread_id();
            std::vector<Entry>& buf = tbuf[tid];
            std::vector<Entry> acc;
#pragma omp for schedule(dynamic, 512)
            for (size_t a = 0; a < next.size(); ++a) {
                const int32_t u = next[a];
                acc.clear();
                int cnt = 0;
                for (int32_t q = GT.ptr[u]; q < GT.ptr[u + 1]; ++q) {
                    const int32_t w = other_end(GT.idx[q], u);
                    if (w < 0) {
                        ++cnt;
                    } else if (layer[w] == d - 1) {
                        ++cnt;
                        acc.insert(acc.end(), rowp[w], rowp[w] + len[w]);
                    }
                }
                std::sort(acc.begin(), acc.end(),
                          [](const Entry& x, const Entry& y) { return x.first < y.first; });
                bthread[a] = tid;
                boff[a] = (int64_t)buf.size();
                size_t k = 0;
                while (k < acc.size()) {
                    double sum = 0.0;
                    const int32_t c = acc[k].first;
                    for (; k < acc.size() && acc[k].first == c; ++k) sum += acc[k].second;
                    buf.emplace_back(c, sum / cnt);
                }
                len[u] = (int32_t)(buf.size() - boff[a]);
            }
        }
        // the buffers are complete: their rows' addresses stay fixed from here on
        for (size_t a = 0; a < next.size(); ++a) rowp[next[a]] = tbuf[bthread[a]].data() + boff[a];
    }
    {
        HostCSR& Pn = out.Pn;
        Pn.nrows = m;
        Pn.ncols = ncn;
        Pn.ptr.assign(m + 1, 0);
        for (int v = 0; v < m; ++v) Pn.ptr[v + 1] = Pn.ptr[v] + len[v];
        Pn.idx.resize(Pn.ptr[m]);
        Pn.val.resize(Pn.ptr[m]);
#pragma omp parallel for schedule(static) num_threads(nth)
        for (int v = 0; v < m; ++v)
            for (int32_t t = 0; t < len[v]; ++t) {
                Pn.idx[Pn.ptr[v] + t] = rowp[v][t].first;
                Pn.val[Pn.ptr[v] + t] = rowp[v][t].second;
            }
    }
    clk.mark("commuting: nodal interp.");
    const HostCSR& Pn = out.Pn;

    // positions in P^T of every entry of P (rows of P sorted by column)
    out.pt_pos.assign(P.nnz(), -1);
#pragma omp parallel for schedule(dynamic, 1024) num_threads(nth)
    for (int c = 0; c < nc; ++c)
        for (int32_t t = PT.ptr[c]; t < PT.ptr[c + 1]; ++t) {
            const int32_t i = PT.idx[t];
            const int32_t* b = P.idx.data() + P.ptr[i];
            const int32_t* e = P.idx.data() + P.ptr[i + 1];
            out.pt_pos[std::lower_bound(b, e, c) - P.idx.data()] = t;
        }
    std::vector<char> ext(n, 0);
    for (const auto& e : cz.edges) ext[e.d1] = ext[e.d2] = 1;
    out.rows.clear();
    for (int i = 0; i < n; ++i)
        if (!ext[i] && P.ptr[i + 1] > P.ptr[i]) out.rows.push_back(i);
    const size_t nr = out.rows.size();
    clk.mark("commuting: P^T positions");

    // local nodes of a row: the coarse nodes its pattern's G_c rows touch, ascending; first into
    // slots of 2 per entry, then compacted
    std::vector<int64_t> slot(nr + 1, 0);
    for (size_t r = 0; r < nr; ++r) slot[r + 1] = slot[r] + 2 * (P.ptr[out.rows[r] + 1] - P.ptr[out.rows[r]]);
    std::vector<int32_t> wide(slot[nr]);
    out.node_ptr.assign(nr + 1, 0);
    clk.mark("commuting: slots");
#pragma omp parallel for schedule(dynamic, 1024) num_threads(nth)
    for (size_t r = 0; r < nr; ++r) {
        const int32_t i = out.rows[r];
        int32_t* nodes = wide.data() + slot[r];
        int k = 0;
        for (int32_t q = P.ptr[i]; q < P.ptr[i + 1]; ++q)
            for (int32_t t = Gc.ptr[P.idx[q]]; t < Gc.ptr[P.idx[q] + 1]; ++t) nodes[k++] = Gc.idx[t];
        std::sort(nodes, nodes + k);
        out.node_ptr[r + 1] = (int32_t)(std::unique(nodes, nodes + k) - nodes);
    }
    int mx = 0;
    for (size_t r = 0; r < nr; ++r) {
        mx = std::max(mx, out.node_ptr[r + 1]);
        out.node_ptr[r + 1] += out.node_ptr[r];
    }
    out.max_nodes = mx;
    clk.mark("commuting: sorted nodes");
    if (mx > 32000) return "a row of the commuting correction touches too many coarse nodes";
    out.t.assign(out.node_ptr[nr], 0.0);
    out.comp.assign(out.node_ptr[nr], -1);
    out.ea.assign(P.nnz(), 0);
    out.eb.assign(P.nnz(), 0);
    clk.mark("commuting: node lists");
#pragma omp parallel num_threads(nth)
    {
        std::vector<int32_t> parent;
        std::vector<char> grounded;
#pragma omp for schedule(dynamic, 1024)
        for (size_t r = 0; r < nr; ++r) {
            const int32_t i = out.rows[r];
            const int32_t* nodes = wide.data() + slot[r];
            const int nl = out.node_ptr[r + 1] - out.node_ptr[r];
            auto loc = [&](int32_t u) { return (int32_t)(std::lower_bound(nodes, nodes + nl, u) - nodes); };
            // t = row i of 2 G P_n on the local nodes
            double* t = out.t.data() + out.node_ptr[r];
            for (int32_t q = G.ptr[i]; q < G.ptr[i + 1]; ++q) {
                const int32_t v = G.idx[q];
                const double g = G.val[q];
                for (int32_t e = Pn.ptr[v]; e < Pn.ptr[v + 1]; ++e) {
                    const int32_t l = loc(Pn.idx[e]);
                    if (l < nl && nodes[l] == Pn.idx[e]) t[l] += 2.0 * g * Pn.val[e];
                }
            }
            // the signed local ends of every entry, and the components of the local graph
            parent.resize(nl);
            std::iota(parent.begin(), parent.end(), 0);
            grounded.assign(nl, 0);
            auto find = [&](int32_t x) {
                while (parent[x] != x) x = parent[x] = parent[parent[x]];
                return x;
            };
            for (int32_t q = P.ptr[i]; q < P.ptr[i + 1]; ++q) {
                const int32_t c = P.idx[q];
                int32_t ends[2] = {-1, -1};
                int ne = 0;
                for (int32_t t2 = Gc.ptr[c]; t2 < Gc.ptr[c + 1] && ne < 2; ++t2) {
                    const int32_t l = loc(Gc.idx[t2]);
                    const int sg = Gc.val[t2] > 0 ? 1 : -1;
                    (ne == 0 ? out.ea[q] : out.eb[q]) = (int16_t)(sg * (l + 1));
                    ends[ne++] = l;
                }
                if (ne == 2) {
                    int32_t x = find(ends[0]), y = find(ends[1]);
                    if (x != y) {
                        if (x > y) std::swap(x, y);
                        parent[y] = x;   // the smaller root stays: a root is its component's first node
                        grounded[x] = grounded[x] | grounded[y];
                    }
                } else if (ne == 1) {
                    grounded[find(ends[0])] = 1;
                }
            }
            int32_t* comp = out.comp.data() + out.node_ptr[r];
            for (int u = 0; u < nl; ++u) {
                const int32_t root = find(u);
                comp[u] = grounded[root] ? -1 : root;
            }
        }
    }
    clk.mark("commuting: row data");
    return "";
}

}  // namespace amgh
