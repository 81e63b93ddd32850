"""Plain FP64 CPU oracle of the fully algebraic H(curl) AMG (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this module; the GPU library never calls it and shares no code with it.  Everything here is written
for reading against the paper (Shen, Brannick, Falgout, Kahl, Schroder, "Nodal Coarsening and Sparse
Ideal Interpolation for H(curl) Problems in Algebraic Multigrid"), not for speed: library primitives
(scipy sparse products, dense LAPACK factorisations, a heap) serve as steps, with no blocking or
fusion beyond what the algorithms state.

Readings of points the paper leaves open (each is repeated where it is used):
  R1 (Sec. 3.1, Eq. sparseP) A_II^{-1} is applied per coarse edge on a local patch: the union of the
     connected components of graph(A_II) touched by the edge's interior A-neighbours if it has at
     most p_max DoFs (exactly P_app, the 2-D situation), else the ring-`ring` interior
     A-neighbourhood of its two exterior DoFs, truncated to p_max in BFS order (ties by index),
     with zero Dirichlet data outside.  Mode "global" solves with the whole A_II.
  R2 (Alg. 2) "classical C/F splitting" is the Ruge-Stueben first pass with measure
     |N(i) & U| + 2 |N(i) & F|, largest measure first, ties to the smallest index; nodes without
     any neighbour are F.
  R3 (Sec. 4.1, Alg. 2) the nodal graph joins two gradient modes (columns of G) when either is a
     classical Ruge-Stueben strong connection of the other in A_G = G^T A G
     (-a_ij >= 0.25 max_{k != i} -a_ik), and joins any two nodes that share an edge of G~ (the
     nearest neighbours the distance-two paths run through; the only links of the artificial
     boundary nodes, which are not gradient modes).  In 2-D this graph equals the symbolic pattern
     of A_G~ on every level; in 3-D the symbolic pattern of coarse levels reaches distance two and
     leaves no distance-two paths.  The Galerkin pattern of P^T A P is symbolic (no dropping).
  R4 (Alg. 3) the middle node k must be a mutual neighbour of i and j in the nodal graph and share
     an edge (a row of G~) with each of them; the smallest such k not yet used is taken.
  R5 (Alg. 3 vs Sec. 3) R has entries +-1 (signs s1 = G~(DoF1,k), s2 = -G~(DoF2,k), so that
     r^T G~ = e_j - e_i); coarse edges are numbered in creation order.
  R6 (Alg. 1) one artificial column per boundary edge-row.
  R7 (Sec. 5, OSS-l1) smoother blocks are node stars {e : G_l(e,j) != 0} of the level's gradient;
     stars are coloured greedily (ascending j, smallest free colour) on the graph "an entry of
     A_l couples the two stars"; a pre-step is multiplicative Schwarz over colours 1..C then
     C-1..1 (colour C once: its exact block solves make a repeat an identity) followed by
     l1-Jacobi with D_ii = sum_j |a_ij|; the post-step is the adjoint (l1-Jacobi first).
  R8 (Eq. Gc) I_C keeps the nonzero columns of R G, in ascending order.
  R9 (Sec. 5) coarsening stops when n <= coarse_size, at max_levels, when a level yields no
     coarse edge, or when n_c > 0.9 n.
  R10 (Eq. commuting; interp="constrained", the 3-D localisation the paper leaves open) the
     nodal interpolation P_n maps the columns of G~ to the coarse nodes: a coarse node (a column
     kept by I_C) is injected; the middle node k of a pair (i, k, j) takes half of each of its
     two ends (an end that is not a coarse node, i.e. a boundary node, counts as zero); every
     other node outside B, in breadth-first layers of the incidence graph from those nodes, takes
     the mean over its neighbours in the previous layer and in the boundary nodes B (zero).
     On the refinement of a hex mesh this is trilinear interpolation.
  R11 (Eq. sparseP with Eq. commuting; interp="constrained") with R's rows (+-1, +-1) the
     exterior rows R^T satisfy P G_c = 2 G P_n (a half edge carries half of its coarse edge's
     difference); every interior row p_i of the local extension (R1) is replaced by the nearest
     row on the same pattern S_i (Euclidean norm) that satisfies row i of that relation, in the
     least-squares sense where none on S_i does: p_i + (t_i - p_i C_i) C_i^+, with C_i the rows
     S_i of G_c and t_i row i of 2 G P_n.
"""
import heapq

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph
import scipy.sparse.linalg as spla

# ----------------------------------------------------------------------------------------------
# sparse-pattern helpers
# ----------------------------------------------------------------------------------------------


def pattern(M):
    """Binary (all-ones) copy of the stored pattern of M, CSR."""
    P = sp.csr_matrix(M, copy=True)
    P.data = np.ones_like(P.data, dtype=np.float64)
    return P


def symbolic_product(*mats):
    """Pattern of the product of the given matrices' patterns.  With all-ones factors no sum can
    cancel, so this is the symbolic sparsity pattern (R3)."""
    out = pattern(mats[0])
    for M in mats[1:]:
        out = pattern(out @ pattern(M))
    out.sort_indices()
    return out


def values_on_pattern(pat, vals):
    """CSR with the pattern of `pat` and the values of `vals` (0 where vals stores nothing)."""
    pat = sp.csr_matrix(pat)
    pat.sort_indices()
    v = sp.coo_matrix(vals)
    nc = pat.shape[1]
    rows = np.repeat(np.arange(pat.shape[0]), np.diff(pat.indptr))
    keys = rows.astype(np.int64) * nc + pat.indices
    vkeys = v.row.astype(np.int64) * nc + v.col
    order = np.argsort(vkeys)
    vkeys, vdata = vkeys[order], v.data[order]
    pos = np.searchsorted(vkeys, keys)
    pos_c = np.minimum(pos, max(len(vkeys) - 1, 0))
    hit = (pos < len(vkeys)) & (vkeys[pos_c] == keys) if len(vkeys) else np.zeros(len(keys), bool)
    data = np.zeros(len(keys))
    data[hit] = vdata[pos_c[hit]]
    if len(vkeys) and not np.all(np.isin(vkeys, keys)):
        raise ValueError("values outside the symbolic pattern")
    return sp.csr_matrix((data, pat.indices.copy(), pat.indptr.copy()), shape=pat.shape)


def neighbours(S):
    """Off-diagonal adjacency lists (sorted int arrays) of a square pattern."""
    S = sp.csr_matrix(S)
    S.sort_indices()
    out = []
    for i in range(S.shape[0]):
        row = S.indices[S.indptr[i]:S.indptr[i + 1]]
        out.append(row[row != i])
    return out


# ----------------------------------------------------------------------------------------------
# Alg. 1: augment G with boundary-node columns
# ----------------------------------------------------------------------------------------------


def augment_G(G):
    """Alg. 1 (Sec. 4.1): for every row of G with exactly one nonzero delta append a column with
    -delta in that row (R6).  Returns (G~, B) with B the appended column indices m..m+k-1."""
    G = sp.csr_matrix(G)
    G.sort_indices()
    n, m = G.shape
    nnz_row = np.diff(G.indptr)
    extra_rows, extra_vals = [], []
    for i in range(n):
        if nnz_row[i] == 1:
            delta = G.data[G.indptr[i]]
            extra_rows.append(i)
            extra_vals.append(-delta)
    k = len(extra_rows)
    ext = sp.csr_matrix((extra_vals, (extra_rows, np.arange(k))), shape=(n, k))
    Gt = sp.csr_matrix(sp.hstack([G, ext]))
    Gt.sort_indices()
    return Gt, np.arange(m, m + k)


# ----------------------------------------------------------------------------------------------
# Sec. 4.1: nodal dual operator graph and edge incidence
# ----------------------------------------------------------------------------------------------


def nodal_graph(A, Gt, nB=0, strength="classical", theta=0.25):
    """Neighbour lists of the nodal graph of A_G~ = G~^T A G~ (Sec. 4.1), reading R3.

    strength="classical": between two gradient modes (original columns of G) j is a neighbour
    of i when -a_ij >= theta max_{k != i}(-a_ik) in A_G~ (Ruge-Stueben strength of a "classical
    C/F splitting"), symmetrised; in addition any two nodes sharing an edge of G~ are
    neighbours (the nearest neighbours the distance-two paths of Alg. 3 run through).  The last
    nB columns (the artificial boundary nodes of Alg. 1) are not gradient modes, so they join the
    graph through shared edges only.  strength="symbolic": the whole symbolic pattern of A_G~."""
    Mp = symbolic_product(Gt.T.tocsr(), Gt)
    if strength == "symbolic":
        return neighbours(symbolic_product(Gt.T.tocsr(), A, Gt))
    nn = Gt.shape[1]
    m = nn - nB
    G = sp.csr_matrix(Gt)[:, :m]
    AG = sp.csr_matrix(G.T @ sp.csr_matrix(A) @ G)
    AG.sort_indices()
    rows = np.repeat(np.arange(m), np.diff(AG.indptr))
    off = AG.indices != rows
    neg = np.where(off, -AG.data, -np.inf)
    rowmax = np.full(m, -np.inf)
    np.maximum.at(rowmax, rows, neg)
    strong = off & (rowmax[rows] > 0) & (neg >= theta * rowmax[rows])
    S = sp.csr_matrix((np.ones(int(strong.sum())), (rows[strong], AG.indices[strong])),
                      shape=(nn, nn))
    return neighbours(pattern(S + S.T + Mp))


def incidence_graph(Gt):
    """M(i): nodes that share a row (an edge) of G~ with node i."""
    return neighbours(symbolic_product(Gt.T.tocsr(), Gt))


# ----------------------------------------------------------------------------------------------
# Alg. 2: nodal C/F splitting with prescribed boundary nodes
# ----------------------------------------------------------------------------------------------
U_, C_, F_ = 0, 1, 2


def nodal_cf(N, B):
    """Alg. 2 (Sec. 4.1).  C starts as B, F as the union of N(b) over b in B (minus B), then the
    Ruge-Stueben first pass (R2) splits the rest.  Returns (c_G = C minus B, f_G, state)."""
    nn = len(N)
    state = np.full(nn, U_, dtype=np.int8)
    state[B] = C_
    for b in B:
        for j in N[b]:
            if state[j] == U_:
                state[j] = F_
    for i in range(nn):
        if state[i] == U_ and len(N[i]) == 0:
            state[i] = F_
    lam = np.zeros(nn, dtype=np.int64)
    heap = []
    for i in range(nn):
        if state[i] == U_:
            lam[i] = sum(1 if state[j] == U_ else (2 if state[j] == F_ else 0) for j in N[i])
            heap.append((-lam[i], i))
    heapq.heapify(heap)
    while heap:
        negl, i = heapq.heappop(heap)
        if state[i] != U_ or -negl != lam[i]:
            continue                       # stale entry
        state[i] = C_
        new_f = [j for j in N[i] if state[j] == U_]
        for j in new_f:
            state[j] = F_
        for j in new_f:
            for l in N[j]:
                if state[l] == U_:
                    lam[l] += 1
                    heapq.heappush(heap, (-lam[l], l))
    isB = np.zeros(nn, dtype=bool)
    isB[B] = True
    cG = np.flatnonzero((state == C_) & ~isB)
    fG = np.flatnonzero(state == F_)
    return cG, fG, state


# ----------------------------------------------------------------------------------------------
# Alg. 3: pairing fine edges into coarse edges along distance-two paths
# ----------------------------------------------------------------------------------------------


def edge_lookup(Gt):
    """(min node, max node) -> smallest row of G~ holding both (rows with two nonzeros)."""
    Gt = sp.csr_matrix(Gt)
    table = {}
    for r in range(Gt.shape[0]):
        cols = Gt.indices[Gt.indptr[r]:Gt.indptr[r + 1]]
        if len(cols) == 2:
            key = (int(min(cols)), int(max(cols)))
            if key not in table:
                table[key] = r
    return table


def match_coarse_edges(Gt, N, M, cG, B, ndof):
    """Alg. 3 (Sec. 4.2): for coarse pairs i < j of c_G u B, not both in B, at distance two in the
    nodal graph, take the smallest middle node k (R4) not in K, pair DoF1 = edge(i,k) and
    DoF2 = edge(k,j) into one row of R with signs (R5), remove them from dof and add k to K.

    Returns a list of (dof1, s1, dof2, s2, i, k, j) in creation order."""
    Gt = sp.csr_matrix(Gt)
    nn = len(N)
    Cp = np.union1d(cG, B)
    isB = np.zeros(nn, dtype=bool)
    isB[B] = True
    inC = np.zeros(nn, dtype=bool)
    inC[Cp] = True
    Nset = [set(a.tolist()) for a in N]
    Mset = [set(a.tolist()) for a in M]
    # pairs at distance <= 2 inside C' (pattern of N N restricted to C')
    Npat = sp.csr_matrix((np.ones(sum(len(a) for a in N)),
                          np.concatenate(N) if nn else np.zeros(0, int),
                          np.concatenate([[0], np.cumsum([len(a) for a in N])])), shape=(nn, nn))
    D2 = symbolic_product(Npat, Npat)
    edge = edge_lookup(Gt)
    dof_free = np.ones(ndof, dtype=bool)
    K = set()
    out = []
    for i in Cp:
        row = D2.indices[D2.indptr[i]:D2.indptr[i + 1]]
        for j in row:
            if j <= i or not inC[j]:
                continue
            if isB[i] and isB[j]:
                continue                                   # (i, j) not both in B
            if j in Nset[i]:
                continue                                   # neighbours, not distance two
            cands = sorted((Nset[i] & Nset[j] & Mset[i] & Mset[j]) - {int(i), int(j)})
            k = next((c for c in cands if c not in K), None)
            if k is None:
                continue
            d1 = edge[(min(i, k), max(i, k))]
            d2 = edge[(min(k, j), max(k, j))]
            assert dof_free[d1] and dof_free[d2]
            s1 = Gt[d1, k]
            s2 = -Gt[d2, k]
            dof_free[d1] = dof_free[d2] = False
            K.add(k)
            out.append((int(d1), float(s1), int(d2), float(s2), int(i), int(k), int(j)))
    return out


def restriction(edges, ndof):
    """R (n_c x n): row c has s1 at DoF1 and s2 at DoF2 (R5)."""
    nc = len(edges)
    rows = np.repeat(np.arange(nc), 2)
    cols = np.array([[e[0], e[2]] for e in edges], dtype=np.int64).ravel()
    vals = np.array([[e[1], e[3]] for e in edges]).ravel()
    R = sp.csr_matrix((vals, (rows, cols)), shape=(nc, ndof))
    R.sort_indices()
    return R


def coarse_gradient(G, R):
    """Eq. Gc: G_c = R G I_C, I_C keeping the nonzero columns of R G (R8).
    Returns (G_c, kept column ids of G)."""
    RG = sp.csr_matrix(R @ G)
    RG.eliminate_zeros()
    keep = np.unique(RG.indices)
    Gc = sp.csr_matrix(RG[:, keep])
    Gc.sort_indices()
    return Gc, keep


# ----------------------------------------------------------------------------------------------
# Eq. sparseP: interior harmonic extension of the coarse variables
# ----------------------------------------------------------------------------------------------


def interior_patches(A, edges, ndof, p_max=128, ring=1):
    """Local patch (sorted interior DoFs) of every coarse edge, reading R1."""
    A = sp.csr_matrix(A)
    ext = np.zeros(ndof, dtype=bool)
    for e in edges:
        ext[e[0]] = ext[e[2]] = True
    interior = np.flatnonzero(~ext)
    AII = pattern(A[interior][:, interior])
    ncomp, comp_local = csgraph.connected_components(AII, directed=False)
    comp = np.full(ndof, -1)
    comp[interior] = comp_local
    comp_size = np.bincount(comp_local, minlength=ncomp)
    members = [[] for _ in range(ncomp)]
    for d in interior:
        members[comp[d]].append(d)
    nbr = lambda d: A.indices[A.indptr[d]:A.indptr[d + 1]]
    patches = []
    for e in edges:
        seeds = sorted(set(int(c) for d in (e[0], e[2]) for c in nbr(d) if not ext[c]))
        comps = sorted(set(comp[s] for s in seeds))
        if sum(comp_size[c] for c in comps) <= p_max:
            patch = sorted(d for c in comps for d in members[c])
        else:
            order = list(seeds)
            seen = set(seeds)
            level = seeds
            for _ in range(ring - 1):
                nxt = sorted(set(int(c) for d in level for c in nbr(d)
                                 if not ext[c] and int(c) not in seen))
                order += nxt
                seen.update(nxt)
                level = nxt
            patch = sorted(order[:p_max])
        patches.append(np.array(patch, dtype=np.int64))
    return patches


def _local_columns(task):
    """Columns c0, c0+1, ... of Eq. sparseP with R1 (one run of coarse edges and their patches):
    R^T e_c on the pair, -A_pp^{-1} A_{p,E_c} r_c on the patch.  Returns (rows, cols, vals)."""
    A, c0, edges, patches = task
    rows, cols, vals = [], [], []
    for c, (e, p) in enumerate(zip(edges, patches), c0):
        d1, s1, d2, s2 = e[0], e[1], e[2], e[3]
        rows += [d1, d2]
        cols += [c, c]
        vals += [s1, s2]
        if len(p):
            App = A[p][:, p].toarray()
            rhs = (A[p][:, [d1]].toarray().ravel() * s1 + A[p][:, [d2]].toarray().ravel() * s2)
            x = -sla.cho_solve(sla.cho_factor(App, lower=True), rhs)
            rows += p.tolist()
            cols += [c] * len(p)
            vals += x.tolist()
    return rows, cols, vals


def _runs(count, nchunks):
    b = np.linspace(0, count, max(1, nchunks) + 1).astype(int)
    return list(zip(b[:-1], b[1:]))


def interpolation_local(A, edges, patches, ndof, pmap=map, nchunks=1):
    """Eq. sparseP with R1: column c = R^T e_c - S_p A_pp^{-1} A_{p,E_c} r_c on patch p.  The
    columns are independent; `pmap` (a map over runs of columns, e.g. a process pool's) may
    compute the nchunks runs in parallel; the result does not depend on it."""
    A = sp.csr_matrix(A)
    rows, cols, vals = [], [], []
    for r, c, v in pmap(_local_columns, [(A, a, edges[a:b], patches[a:b]) for a, b in _runs(len(edges), nchunks)]):
        rows += r
        cols += c
        vals += v
    P = sp.csr_matrix((vals, (rows, cols)), shape=(ndof, len(edges)))
    P.sort_indices()
    return P


def interpolation_global(A, edges, ndof):
    """Eq. sparseP exactly: P = (I - S_I A_II^{-1} S_I^T A) R^T, for small problems only."""
    A = sp.csc_matrix(A)
    R = restriction(edges, ndof)
    ext = np.zeros(ndof, dtype=bool)
    for e in edges:
        ext[e[0]] = ext[e[2]] = True
    I = np.flatnonzero(~ext)
    RT = R.T.tocsc()
    rhs = (A[I] @ RT).toarray()
    X = -spla.splu(A[I][:, I].tocsc()).solve(rhs) if len(I) else np.zeros((0, len(edges)))
    P = RT.toarray()
    P[I] = X
    return sp.csr_matrix(P)


# ----------------------------------------------------------------------------------------------
# Eq. commuting: the local extension corrected to commute with a nodal interpolation (R10, R11)
# ----------------------------------------------------------------------------------------------


def nodal_interpolation(Gt, B, edges, coarse_nodes):
    """R10: P_n (columns of G~ x coarse nodes).  Layer 0 holds the coarse nodes (injected) and
    the middle nodes of the pairs (half of each coarse end); layer d + 1 holds the nodes outside B
    first reached from layer d in the incidence graph, each the mean of its neighbours in layer d
    and in B (the boundary nodes, zero).  Nodes never reached keep zero rows."""
    Gt = sp.csr_matrix(Gt)
    nn = Gt.shape[1]
    nc = len(coarse_nodes)
    col = np.full(nn, -1, dtype=np.int64)
    col[coarse_nodes] = np.arange(nc)
    layer = np.full(nn, -1, dtype=np.int64)
    layer[coarse_nodes] = 0
    rows, cols, vals = list(coarse_nodes), list(range(nc)), [1.0] * nc
    for e in edges:
        i, k, j = e[4], e[5], e[6]
        if k < 0:
            continue
        layer[k] = 0
        for end in (i, j):
            if end >= 0 and col[end] >= 0:
                rows.append(k)
                cols.append(col[end])
                vals.append(0.5)
    Pn = sp.csr_matrix((vals, (rows, cols)), shape=(nn, nc))
    nbr = incidence_graph(Gt)
    Adj = sp.csr_matrix((np.ones(sum(len(a) for a in nbr)), np.concatenate(nbr) if nn else np.zeros(0, int),
                         np.concatenate([[0], np.cumsum([len(a) for a in nbr])])), shape=(nn, nn))
    isB = np.zeros(nn, dtype=bool)
    isB[B] = True
    d = 0
    while True:
        reached = Adj @ ((layer == d) & ~isB).astype(np.float64)
        nxt = np.flatnonzero((reached > 0) & (layer < 0) & ~isB)
        if len(nxt) == 0:
            break
        d += 1
        layer[nxt] = d
        eligible = ((layer == d - 1) | isB).astype(np.float64)
        Wn = sp.csr_matrix(Adj[nxt] @ sp.diags(eligible))
        Wn = sp.csr_matrix(sp.diags(1.0 / np.asarray(Wn.sum(axis=1)).ravel()) @ Wn)
        place = sp.csr_matrix((np.ones(len(nxt)), (nxt, np.arange(len(nxt)))), shape=(nn, len(nxt)))
        Pn = sp.csr_matrix(Pn + place @ (Wn @ Pn))
    Pn.sort_indices()
    return Pn


def interpolation_constrained(P, G, Gc, Pn, edges):
    """R11: every interior row of P moved, on its own pattern, to the nearest row satisfying
    row i of P G_c = 2 G P_n (least squares where it cannot); exterior rows kept."""
    P = sp.csr_matrix(P, copy=True)
    P.sort_indices()
    G = sp.csr_matrix(G)
    m = G.shape[1]
    T = sp.csr_matrix(2.0 * (G @ sp.csr_matrix(Pn)[:m]))
    Gc = sp.csr_matrix(Gc)
    ext = np.zeros(P.shape[0], dtype=bool)
    for e in edges:
        ext[e[0]] = ext[e[2]] = True
    data = P.data.copy()
    for i in np.flatnonzero(~ext):
        a, b = P.indptr[i], P.indptr[i + 1]
        if a == b:
            continue
        C = Gc[P.indices[a:b]]
        nodes = np.union1d(C.indices, T.indices[T.indptr[i]:T.indptr[i + 1]])
        Cd = C[:, nodes].toarray()
        t = T[i][:, nodes].toarray().ravel()
        p0 = P.data[a:b]
        # C_i is a +-1 incidence block whose rank is structural: its nonzero singular values are
        # at least 1/k for k nodes, its zero ones come out of the SVD as rounding noise (up to
        # ~1e-13 sigma_max), so the pseudo-inverse cuts at 1e-8 sigma_max
        data[a:b] = p0 + (t - p0 @ Cd) @ np.linalg.pinv(Cd, rcond=1e-8)
    return sp.csr_matrix((data, P.indices.copy(), P.indptr.copy()), shape=P.shape)


def galerkin(A, P):
    """A_c = P^T A P (Eq. tl) on the symbolic pattern (R3)."""
    Pt = sp.csr_matrix(P.T)
    pat = symbolic_product(Pt, A, P)
    return values_on_pattern(pat, Pt @ (A @ P))


# ----------------------------------------------------------------------------------------------
# Smoother: OSS-l1 on node stars (reading R7)
# ----------------------------------------------------------------------------------------------


def stars(G):
    """Star of node j: the rows e with G(e, j) != 0, ascending."""
    Gc = sp.csc_matrix(G)
    Gc.sort_indices()
    return [Gc.indices[Gc.indptr[j]:Gc.indptr[j + 1]].copy() for j in range(G.shape[1])]


def colour_stars(A, G):
    """Greedy colouring (ascending j, smallest free colour) of the star conflict graph: j ~ j' when
    an entry of A couples star j and star j' (a shared DoF included)."""
    S = neighbours(symbolic_product(sp.csr_matrix(G.T), A, G))
    ns = len(S)
    colour = np.full(ns, -1, dtype=np.int64)
    for j in range(ns):
        used = set(colour[S[j]].tolist())
        c = 0
        while c in used:
            c += 1
        colour[j] = c
    return colour


def _inverses(task):
    A, blocks = task
    return [np.linalg.inv(A[b][:, b].toarray()) for b in blocks]


def star_inverses(A, st, pmap=map, nchunks=1):
    """Dense inverses of the star blocks A[B_j, B_j] (independent; `pmap` as in
    interpolation_local)."""
    A = sp.csr_matrix(A)
    out = []
    for part in pmap(_inverses, [(A, st[a:b]) for a, b in _runs(len(st), nchunks)]):
        out += part
    return out


def l1_diagonal(A):
    return np.asarray(abs(sp.csr_matrix(A)).sum(axis=1)).ravel()


def _schwarz_colour(L, c, f, x):
    r = f - L["A"] @ x
    for j in L["colour_members"][c]:
        b = L["stars"][j]
        x[b] += L["inv"][j] @ r[b]


def _colour_sequence(ncol):
    return list(range(ncol)) + list(range(ncol - 2, -1, -1))


def smooth_pre(L, f, x):
    """Symmetric multiplicative Schwarz over colours, then l1-Jacobi (R7)."""
    for c in _colour_sequence(L["ncolours"]):
        _schwarz_colour(L, c, f, x)
    x += (f - L["A"] @ x) / L["l1"]
    return x


def smooth_post(L, f, x):
    """Adjoint of smooth_pre: l1-Jacobi, then the symmetric colour sweep."""
    x += (f - L["A"] @ x) / L["l1"]
    for c in _colour_sequence(L["ncolours"]):
        _schwarz_colour(L, c, f, x)
    return x


# ----------------------------------------------------------------------------------------------
# Hierarchy (Sec. 4 two-level setup, recursed; Sec. 5 limits)
# ----------------------------------------------------------------------------------------------


# ----------------------------------------------------------------------------------------------
# Sec. 3 and Sec. 5: refinement-based coarse variables ("Ref") and geometric Nedelec
# interpolation ("Geo") on the structured n^3 hex mesh
# ----------------------------------------------------------------------------------------------


def hex_numbering(n):
    """Interior edge and node ids of the n^3 hex mesh of the unit cube, as the inputs number them:
    x-edges, then y, then z, each lexicographic by start node (i fastest), oriented +axis; edges
    lying in a boundary face and boundary nodes are eliminated (id -1).  Returns (edge_id(d, i, j,
    k), node_id(i, j, k)) for integer node coordinates 0..n."""
    m = n - 1
    nx = n * m * m

    def edge_id(d, i, j, k):
        if d == 0:
            ok = 0 <= i < n and 1 <= j <= m and 1 <= k <= m
            return i + n * ((j - 1) + m * (k - 1)) if ok else -1
        if d == 1:
            ok = 1 <= i <= m and 0 <= j < n and 1 <= k <= m
            return nx + (i - 1) + m * (j + n * (k - 1)) if ok else -1
        ok = 1 <= i <= m and 1 <= j <= m and 0 <= k < n
        return 2 * nx + (i - 1) + m * ((j - 1) + m * k) if ok else -1

    def node_id(i, j, k):
        ok = 1 <= i <= m and 1 <= j <= m and 1 <= k <= m
        return (i - 1) + m * ((j - 1) + m * (k - 1)) if ok else -1

    return edge_id, node_id


def refinement_edges(n):
    """Sec. 3: the coarse variables follow the geometric refinement of the n^3 mesh (n even).  Every
    interior edge of the (n/2)^3 coarse mesh, in the coarse mesh's own numbering, is the pair of
    its two fine halves: DoF1 the half at its tail, DoF2 the half at its head, both oriented like
    the coarse edge, so the row of R is (+1, +1) (the orthogonal complement of the middle node's
    gradient column, signs following G).  Returns (dof1, s1, dof2, s2, i, k, j) with i, k, j the
    tail, middle and head node ids (-1 for a boundary node)."""
    if n % 2 or n < 2:
        raise ValueError("refinement needs an even mesh size")
    N = n // 2
    fe, fn = hex_numbering(n)
    ce, _ = hex_numbering(N)
    steps = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    out = {}
    for d in range(3):
        a, b, c = steps[d]
        for K in range(N + 1):
            for J in range(N + 1):
                for I in range(N + 1):
                    cid = ce(d, I, J, K)
                    if cid < 0:
                        continue
                    x, y, z = 2 * I, 2 * J, 2 * K
                    d1 = fe(d, x, y, z)
                    d2 = fe(d, x + a, y + b, z + c)
                    out[cid] = (d1, 1.0, d2, 1.0, fn(x, y, z), fn(x + a, y + b, z + c),
                                fn(x + 2 * a, y + 2 * b, z + 2 * c))
    return [out[c] for c in range(len(out))]


def interpolation_geometric(n, edges, ndof):
    """Geometric Nedelec interpolation ("Geo", Sec. 5) of the (n/2)^3 mesh's edge space into the
    n^3 mesh's, scaled by 2 so that its rows on the coarse edges' halves are R^T (Eq. sparseP's
    exterior rows).  A coarse edge's basis function points along the edge and decays linearly to
    zero one coarse cell away across it; a fine edge parallel to it at transverse offsets (dy, dz)
    in fine steps (-1, 0, 1) takes the value of that hat product at the fine edge, 1, 1/2 or 1/4,
    times the ratio of the line integrals (fine over coarse length, 1/2), times 2; fine edges across
    the coarse edge get 0."""
    fe, _ = hex_numbering(n)
    steps = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    N = n // 2
    ce, _ = hex_numbering(N)
    rows, cols, vals = [], [], []
    # the start node of every coarse edge, from its id
    starts = {}
    for d in range(3):
        for K in range(N + 1):
            for J in range(N + 1):
                for I in range(N + 1):
                    cid = ce(d, I, J, K)
                    if cid >= 0:
                        starts[cid] = (d, I, J, K)
    hat = {-1: 0.5, 0: 1.0, 1: 0.5}
    for c in range(len(edges)):
        d, I, J, K = starts[c]
        a, b, cc = steps[d]
        t1, t2 = [ax for ax in range(3) if ax != d]
        for half in (0, 1):
            base = [2 * I + half * a, 2 * J + half * b, 2 * K + half * cc]
            for o1 in (-1, 0, 1):
                for o2 in (-1, 0, 1):
                    q = list(base)
                    q[t1] += o1
                    q[t2] += o2
                    e = fe(d, *q)
                    if e >= 0:
                        rows.append(e)
                        cols.append(c)
                        vals.append(hat[o1] * hat[o2])
    P = sp.csr_matrix((vals, (rows, cols)), shape=(ndof, len(edges)))
    P.sort_indices()
    return P


def geometric_patches(n, edges, ndof):
    """Interior support of every column of the geometric interpolation (the fine edges parallel to
    the coarse edge other than its two halves), sorted."""
    Pg = interpolation_geometric(n, edges, ndof).tocsc()
    out = []
    for c, e in enumerate(edges):
        rows = Pg.indices[Pg.indptr[c]:Pg.indptr[c + 1]]
        out.append(np.array(sorted(r for r in rows if r not in (e[0], e[2])), dtype=np.int64))
    return out


def coarsen(A, G, interp="local", p_max=128, ring=1, strength="classical", theta=0.25, pmap=map, nchunks=1,
            splitting="algebraic", mesh_n=None):
    """One application of the two-level setup.  splitting="algebraic" (Sec. 4): augment G
    (Alg. 1), split the nodal dual operator (Alg. 2), pair edges (Alg. 3).  splitting="refinement"
    (Sec. 3): the pairs of the geometric refinement of the mesh_n^3 hex mesh.  Then interpolate
    (Eq. sparseP; interp="geometric": the geometric Nedelec interpolation instead;
    interp="constrained": Eq. sparseP's local extension corrected to commute, R10-R11) and form
    G_c (Eq. Gc)."""
    A = sp.csr_matrix(A)
    G = sp.csr_matrix(G)
    ndof = A.shape[0]
    if splitting == "refinement":
        edges = refinement_edges(mesh_n)
        keep_nodes = sorted({e[4] for e in edges if e[4] >= 0} | {e[6] for e in edges if e[6] >= 0})
        cG = np.array(keep_nodes, dtype=np.int64)
        fG = np.setdiff1d(np.arange(G.shape[1]), cG)
        out = dict(Gt=G, B=np.zeros(0, dtype=np.int64), cG=cG, fG=fG, edges=edges)
    else:
        if interp == "geometric":
            raise ValueError("the geometric interpolation needs the refinement splitting")
        Gt, B = augment_G(G)
        N = nodal_graph(A, Gt, nB=len(B), strength=strength, theta=theta)
        M = incidence_graph(Gt)
        cG, fG, state = nodal_cf(N, B)
        edges = match_coarse_edges(Gt, N, M, cG, B, ndof)
        out = dict(Gt=Gt, B=B, cG=cG, fG=fG, edges=edges)
    if not edges:
        return out
    R = restriction(edges, ndof)
    Gc, keep = coarse_gradient(G, R)
    if interp == "global":
        patches = None
        P = interpolation_global(A, edges, ndof)
    elif interp == "geometric":
        patches = geometric_patches(mesh_n, edges, ndof)
        P = interpolation_geometric(mesh_n, edges, ndof)
    else:
        patches = interior_patches(A, edges, ndof, p_max=p_max, ring=ring)
        P = interpolation_local(A, edges, patches, ndof, pmap=pmap, nchunks=nchunks)
    if interp == "constrained":
        Gn, Bn = (out["Gt"], out["B"]) if splitting != "refinement" else augment_G(G)
        Pn = nodal_interpolation(Gn, Bn, edges, keep)
        out["Pn"] = Pn
        P = interpolation_constrained(P, G, Gc, Pn, edges)
    out.update(R=R, Gc=Gc, coarse_nodes=keep, patches=patches, P=P)
    return out


def smoother_level(A, G, pmap=map, nchunks=1):
    A = sp.csr_matrix(A)
    st = stars(G)
    colour = colour_stars(A, G)
    ncol = int(colour.max()) + 1 if len(colour) else 0
    return dict(A=A, stars=st, colour=colour, ncolours=ncol,
                colour_members=[np.flatnonzero(colour == c) for c in range(ncol)],
                inv=star_inverses(A, st, pmap=pmap, nchunks=nchunks), l1=l1_diagonal(A))


def setup(A, G, coarse_size=100, max_levels=20, interp="local", p_max=128, ring=1,
          stall_ratio=0.9, strength="classical", theta=0.25, pmap=map, nchunks=1, splitting="algebraic",
          mesh_n=None):
    """Build the multilevel hierarchy (R9).  Returns a list of level dicts; every level but the
    last carries P, the last carries the dense Cholesky factor of its matrix.  pmap / nchunks
    spread the independent local solves and star inverses over a parallel map (same result).
    splitting="refinement" (with mesh_n, the hex mesh's intervals per side) coarsens by geometric
    refinement, halving the mesh per level while it stays even."""
    A = sp.csr_matrix(A)
    A.sort_indices()
    G = sp.csr_matrix(G)
    levels = []
    while True:
        n = A.shape[0]
        L = smoother_level(A, G, pmap=pmap, nchunks=nchunks)
        L["G"] = G
        levels.append(L)
        if n <= coarse_size or len(levels) == max_levels:
            break
        if splitting == "refinement" and (mesh_n is None or mesh_n % 2 or mesh_n < 4):
            break
        cz = coarsen(A, G, interp=interp, p_max=p_max, ring=ring, strength=strength, theta=theta,
                     pmap=pmap, nchunks=nchunks, splitting=splitting, mesh_n=mesh_n)
        L["coarsening"] = cz
        nc = len(cz["edges"])
        if nc == 0 or nc > stall_ratio * n:
            L.pop("coarsening")
            break
        L["P"] = cz["P"]
        A = galerkin(A, cz["P"])
        G = cz["Gc"]
        if splitting == "refinement":
            mesh_n //= 2
    last = levels[-1]
    last["chol"] = sla.cho_factor(last["A"].toarray(), lower=True)
    return levels


def vcycle(H, f, l=0):
    """One V-cycle (Eq. tl recursively): zero start, OSS-l1 pre-step, coarse correction with
    P_l^T and P_l, OSS-l1 post-step; dense Cholesky on the last level."""
    L = H[l]
    if l == len(H) - 1:
        return sla.cho_solve(L["chol"], f)
    x = np.zeros_like(f)
    smooth_pre(L, f, x)
    r = f - L["A"] @ x
    ec = vcycle(H, L["P"].T @ r, l + 1)
    x += L["P"] @ ec
    smooth_post(L, f, x)
    return x


def pcg(H, f, x0=None, tol=1e-8, maxit=500, flexible=False, precond=None):
    """Preconditioned CG to ||r_k|| <= tol ||r_0|| (Sec. 5).  With flexible=True the Polak-Ribiere
    coefficient beta = <z_k+1, r_k+1 - r_k> / <z_k, r_k> (flexible CG).
    Returns (x, iterations, residual history)."""
    A = H[0]["A"]
    B = precond if precond is not None else (lambda r: vcycle(H, r))
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - A @ x
    hist = [np.linalg.norm(r)]
    if hist[0] == 0.0:
        return x, 0, hist
    z = B(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r_old = r
        r = r - alpha * q
        hist.append(np.linalg.norm(r))
        if hist[-1] <= tol * hist[0]:
            return x, it, hist
        z = B(r)
        rz_new = r @ z
        beta = (z @ (r - r_old)) / rz if flexible else rz_new / rz
        p = z + beta * p
        rz = rz_new
    return x, maxit, hist


def amg_iterate(H, f, x0=None, tol=1e-8, maxit=1000):
    """Stand-alone V-cycle iteration x <- x + B(f - A x) (Sec. 5 'AMG' counts)."""
    A = H[0]["A"]
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - A @ x
    hist = [np.linalg.norm(r)]
    for it in range(1, maxit + 1):
        x += vcycle(H, r)
        r = f - A @ x
        hist.append(np.linalg.norm(r))
        if hist[-1] <= tol * hist[0]:
            return x, it, hist
    return x, maxit, hist


def convergence_factor(hist):
    """(||r_k|| / ||r_0||)^(1/k), the factor the paper's tables report."""
    k = len(hist) - 1
    return (hist[-1] / hist[0]) ** (1.0 / k) if k else 0.0


def complexities(H):
    """Operator complexity sum nnz(A_l)/nnz(A_0) and grid complexity sum n_l/n_0."""
    nnz = [L["A"].nnz for L in H]
    n = [L["A"].shape[0] for L in H]
    return sum(nnz) / nnz[0], sum(n) / n[0]


def probe_factor(H, x0, cycles=10):
    """Convergence factor of `cycles` stand-alone V-cycles on A x = 0 from x0 (the quantity that
    decides whether a learned interpolation is kept)."""
    _, _, hist = amg_iterate(H, np.zeros(H[0]["A"].shape[0]), x0=x0, tol=0.0, maxit=cycles)
    return convergence_factor(hist)
