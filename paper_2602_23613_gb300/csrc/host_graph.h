// Host-side graph steps of the algebraic H(curl) setup (Section 4 of the paper): pure C++,
// O(nnz) per step, no CUDA.  Integer/pattern work only, apart from the strength test of the
// nodal C/F splitting, which reads values of G^T A G.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace amgh {

struct HostCSR {
    int nrows = 0, ncols = 0;
    std::vector<int32_t> ptr;   // nrows + 1
    std::vector<int32_t> idx;   // nnz, ascending per row
    std::vector<double> val;    // nnz (empty for a pure pattern)
    int64_t nnz() const { return ptr.empty() ? 0 : ptr.back(); }
};

HostCSR transpose_pattern(const HostCSR& M, bool with_values);
// the same on nthreads OpenMP threads (identical result)
HostCSR transpose_pattern(const HostCSR& M, bool with_values, int nthreads);

struct CoarseEdge {
    int32_t d1, s1, d2, s2;   // fine DoFs and their +-1 signs in the row of R
    int32_t i, k, j;          // coarse end nodes i < j and the middle node k (columns of G~)
};

struct Coarsening {
    int m = 0, nB = 0;                   // original columns of G, artificial boundary columns
    std::vector<int8_t> state;           // per column of G~: 1 = C, 2 = F
    std::vector<CoarseEdge> edges;       // creation order
    std::vector<int32_t> coarse_nodes;   // kept columns of R G, ascending
    HostCSR Gc;                          // n_c x |coarse_nodes|, +-1
    std::vector<int32_t> patch_ptr, patch_idx;   // sorted patch per coarse edge
    HostCSR P;                           // pattern of P (n x n_c); val holds the exterior +-1
    std::vector<int64_t> patch_pos_P;    // position in P.idx of every patch entry
    HostCSR PT;                          // pattern of P^T (n_c x n)
    std::vector<int64_t> patch_pos_PT;   // position in PT.idx of every patch entry
    std::vector<int64_t> ext_pos_P, ext_pos_PT;   // 2 per coarse edge: (d1, c), (d2, c)
    HostCSR AP;                          // symbolic pattern of A P
    HostCSR Ac;                          // symbolic pattern of P^T A P
    // geometric interpolation only: per coarse edge its interior support (sorted) and weights,
    // which then also are the patches
    std::vector<int32_t> geo_ptr, geo_idx;
    std::vector<double> geo_val;
};

struct Params {
    double theta = 0.25;
    int ring = 1;
    int p_max = 128;
    bool symbolic_galerkin = true;   // also form the symbolic AP and P^T A P patterns on the host
};

// pattern of X Y with sorted columns per row (values left empty)
HostCSR symbolic_product(const HostCSR& X, const HostCSR& Y, int nthreads);

// Validate G (rows with 1 or 2 entries of +-1; two entries of opposite sign).  Returns "" if ok.
std::string check_gradient(const HostCSR& G);
std::string check_csr(const HostCSR& M, bool square);

// Alg. 1-3, Eq. sparseP patches, Eq. Gc and the symbolic Galerkin patterns for one level.
// A must carry values (strength test).  Returns "" or an error message.
std::string coarsen_level(const HostCSR& A, const HostCSR& G, const Params& prm, Coarsening& out,
                          int nthreads);

// Section 3's refinement-based pairs on the structured hex mesh with mesh_n intervals per side
// (coarse edges in the (mesh_n/2)^3 mesh's numbering), then the same patches, G_c and patterns;
// with `geometric`, the geometric Nedelec interpolation's supports and weights (geo_*) instead of
// the patches.  Returns "" or an error message.
std::string coarsen_level_refinement(const HostCSR& A, const HostCSR& G, int mesh_n, bool geometric,
                                     const Params& prm, Coarsening& out, int nthreads);

// Eq. commuting: the local extension corrected to commute --------------------------------------
// The nodal interpolation P_n maps the nodes (columns of G) to the coarse nodes: a coarse node is
// injected; the middle node k of a pair (i, k, j) takes half of each end that is a coarse node;
// every other node, in breadth-first layers of the incidence graph from those nodes, takes the
// mean over its neighbours in the previous layer and its boundary edges (one-entry rows of G,
// whose artificial ends carry zero).  With R's rows (+-1, +-1) the exterior rows R^T of P satisfy
// P G_c = 2 G P_n; every interior row of P is moved, on its own pattern, to the nearest row that
// satisfies row i of it (least squares where none does).  Per interior row this holds what the
// device needs for that least-distance problem: its local nodes (the coarse nodes its pattern's
// G_c rows touch, ascending), the target t = row i of 2 G P_n on them, and which local nodes form
// components that no one-ended G_c row of the pattern grounds (their residual is matched only up
// to its mean there, and their first node is left out of the solve).
struct CommutingRows {
    int max_nodes = 0;
    std::vector<int32_t> rows;       // interior rows of P with a nonempty pattern, ascending
    std::vector<int32_t> node_ptr;   // rows.size() + 1: local nodes of each row
    std::vector<double> t;           // per local node: row i of 2 G P_n there
    std::vector<int32_t> comp;       // per local node: first local node of its component when
                                     // nothing grounds the component, else -1
    std::vector<int16_t> ea, eb;     // per entry of P: the local ends of the entry's G_c row as
                                     // (local index + 1) * sign, 0 for none
    std::vector<int32_t> pt_pos;     // per entry of P: its position in P^T
    HostCSR Pn;                      // the nodal interpolation (columns of G x coarse nodes)
};

// needs cz's edges, coarse nodes, G_c and the patterns of P and P^T (from coarsen_level or
// coarsen_level_refinement); returns "" or an error message
std::string commuting_rows(const HostCSR& G, const Coarsening& cz, CommutingRows& out, int nthreads);

// Smoother structure (node stars of G and their colouring) -------------------------------------
struct StarLayout {
    int nstars = 0, ncolours = 0, max_block = 0;
    std::vector<int32_t> star_ptr, star_idx;   // star j = rows e with G(e, j) != 0, ascending
    std::vector<int32_t> colour;               // per star
};

std::string build_stars(const HostCSR& A, const HostCSR& G, StarLayout& out);

}  // namespace amgh
