"""Pins of the oracle's graph steps (Alg. 1-3, Eq. Gc) against brute force, geometry and the
paper's printed complexities."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import amg as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables_1_2.json")


# ---------------------------------------------------------------------------------------------
# brute-force restatements used as independent checks on tiny inputs
# ---------------------------------------------------------------------------------------------
def naive_nodal_cf(N, B):
    """Alg. 2 with an O(n^2) scan for the largest measure (ties to the smallest index)."""
    nn = len(N)
    st = ["U"] * nn
    for b in B:
        st[b] = "C"
    for b in B:
        for j in N[b]:
            if st[j] == "U":
                st[j] = "F"
    for i in range(nn):
        if st[i] == "U" and len(N[i]) == 0:
            st[i] = "F"
    while "U" in st:
        best, bi = -1, -1
        for i in range(nn):
            if st[i] == "U":
                lam = sum(1 if st[j] == "U" else 2 if st[j] == "F" else 0 for j in N[i])
                if lam > best:
                    best, bi = lam, i
        st[bi] = "C"
        for j in N[bi]:
            if st[j] == "U":
                st[j] = "F"
    return np.array([i for i in range(nn) if st[i] == "C" and i not in set(B)])


def naive_match(Gt, N, M, cG, B):
    """Alg. 3 literally: every (i, j) in C' x C' with i < j in ascending order."""
    Gt = sp.csr_matrix(Gt)
    Cp = sorted(set(cG.tolist()) | set(B.tolist()))
    Bs = set(B.tolist())
    Ns = [set(a.tolist()) for a in N]
    Ms = [set(a.tolist()) for a in M]
    K, out = set(), []
    for a, i in enumerate(Cp):
        for j in Cp[a + 1:]:
            if i in Bs and j in Bs:
                continue
            if j in Ns[i] or not (Ns[i] & Ns[j]):
                continue
            cands = sorted((Ns[i] & Ns[j] & Ms[i] & Ms[j]) - {i, j})
            k = next((c for c in cands if c not in K), None)
            if k is None:
                continue
            rows_i = set(Gt[:, i].nonzero()[0])
            rows_k = set(Gt[:, k].nonzero()[0])
            rows_j = set(Gt[:, j].nonzero()[0])
            d1 = min(rows_i & rows_k)
            d2 = min(rows_k & rows_j)
            K.add(k)
            out.append((d1, Gt[d1, k], d2, -Gt[d2, k], i, k, j))
    return out


def _graph_parts(p):
    Gt, B = O.augment_G(p["G"])
    N = O.nodal_graph(p["A"], Gt, nB=len(B))
    M = O.incidence_graph(Gt)
    return Gt, B, N, M


# ---------------------------------------------------------------------------------------------
def test_augment_g_hand_example():
    # rows: (-1,+1 on nodes 0,1), (+1 on node 1 only), (-1 on node 0 only)
    G = sp.csr_matrix(np.array([[-1.0, 1.0], [0.0, 1.0], [-1.0, 0.0]]))
    Gt, B = O.augment_G(G)
    assert B.tolist() == [2, 3]
    np.testing.assert_array_equal(Gt.toarray(), [[-1, 1, 0, 0], [0, 1, -1, 0], [-1, 0, 0, 1]])
    # every row of G~ is a signed incidence row: two entries of opposite sign
    assert np.all(np.asarray(Gt.sum(axis=1)).ravel() == 0)


@pytest.mark.parametrize("maker", [lambda: W.hex_problem(4, W.fields.log_uniform(4, 2), 0.1),
                                   lambda: W.hex_problem(5, 1.0, 1.0),
                                   lambda: W.tri_problem(6, 1.0, 0.01),
                                   lambda: W.quad_problem(7, 1.0, 0.01)])
def test_nodal_cf_and_matching_against_brute_force(maker):
    p = maker()
    Gt, B, N, M = _graph_parts(p)
    cG, fG, state = O.nodal_cf(N, B)
    np.testing.assert_array_equal(cG, naive_nodal_cf(N, B))
    # C is independent (apart from B-B pairs) and every F node has a C neighbour
    C = set(cG.tolist()) | set(B.tolist())
    for i in cG:
        assert not (set(N[i].tolist()) & C)
    for f in fG:
        assert set(N[f].tolist()) & C
    edges = O.match_coarse_edges(Gt, N, M, cG, B, p["ndof"])
    ref = naive_match(Gt, N, M, cG, B)
    assert [(e[0], e[2], e[4], e[5], e[6]) for e in edges] == [(r[0], r[2], r[4], r[5], r[6]) for r in ref]
    assert [(e[1], e[3]) for e in edges] == [(float(r[1]), float(r[3])) for r in ref]


def _hex_node_xyz(n, ids):
    nm = n - 1
    ids = np.asarray(ids)
    return np.stack([ids % nm + 1, (ids // nm) % nm + 1, ids // (nm * nm) + 1], axis=1)


def test_hex8_geometric_coarsening():
    """On the uniform 8^3 hex mesh the algebraic splitting is geometric: coarse nodes are the
    (even)^3 interior nodes and the 108 coarse edges are the interior edges of the 4^3 mesh."""
    n = 8
    p = W.hex_problem(n, 1.0, 1.0)
    cz = O.coarsen(p["A"], p["G"])
    xyz = _hex_node_xyz(n, cz["cG"])
    assert len(cz["cG"]) == 27 and np.all(xyz % 2 == 0)
    edges = cz["edges"]
    assert len(edges) == 3 * 4 * 3 ** 2
    ks = [e[5] for e in edges]
    assert len(set(ks)) == len(ks)                                  # K: one path per middle node
    dofs = [e[0] for e in edges] + [e[2] for e in edges]
    assert len(set(dofs)) == len(dofs)                              # distinct pairing
    R = O.restriction(edges, p["ndof"])
    np.testing.assert_array_equal((R @ R.T).toarray(), 2 * np.eye(len(edges)))
    Gt = cz["Gt"]
    m = p["G"].shape[1]
    for e in edges:
        d1, s1, d2, s2, i, k, j = e
        r = np.zeros(Gt.shape[1])
        r[j] += 1
        r[i] -= 1
        got = (s1 * Gt[d1] + s2 * Gt[d2]).toarray().ravel()
        np.testing.assert_array_equal(got, r)                        # r^T G~ = e_j - e_i
        if j < m:                                                    # interior pair: distance 2 on an axis
            dxyz = np.abs(_hex_node_xyz(n, [j])[0] - _hex_node_xyz(n, [i])[0])
            assert sorted(dxyz.tolist()) == [0, 0, 2]
    Gc = cz["Gc"]
    assert set(np.diff(Gc.indptr).tolist()) <= {1, 2}
    assert np.all(np.abs(Gc.data) == 1)
    assert np.all(np.asarray(Gc.sum(axis=1)).ravel()[np.diff(Gc.indptr) == 2] == 0)


def test_quad_splitting_is_geometric_refinement():
    """Fig. 3 claim: on a uniform square mesh the algebraic splitting equals refinement: coarse
    nodes (even, even), each coarse edge two collinear fine edges, 4 interior DoFs per coarse cell."""
    N = 16
    p = W.quad_problem(N, 1.0, 0.01)
    cz = O.coarsen(p["A"], p["G"])
    Nm = N - 1
    c = cz["cG"]
    assert np.all((c % Nm + 1) % 2 == 0) and np.all((c // Nm + 1) % 2 == 0)
    assert len(c) == (N // 2 - 1) ** 2
    nc = len(cz["edges"])
    assert nc == 2 * (N // 2) * (N // 2 - 1)
    nx = N * Nm
    for d1, s1, d2, s2, i, k, j in cz["edges"]:
        assert (d1 < nx) == (d2 < nx)                                # collinear pair
    assert p["ndof"] - 2 * nc == 4 * (N // 2) ** 2                   # 4 interior DoFs per cell


@pytest.mark.parametrize("table,L", [("table1", 4), ("table1", 5), ("table2", 4)])
def test_paper_complexities_exact(table, L):
    """Operator/grid complexities and level counts of Tables 1-2 (Alg) follow from the structure
    alone; the oracle reproduces the printed values."""
    g = next(r for r in json.load(open(GOLDEN))[table] if r["L"] == L)
    N = 2 ** L
    ne = 2 * N * N
    if table == "table1":
        alpha = np.ones(ne)
    else:
        col = (np.arange(ne) // 2) % N
        alpha = np.where(col % 2 == 0, 10.0, 0.1)
    p = W.tri_problem(N, alpha, 0.01)
    assert p["ndof"] == g["n"]
    H = O.setup(p["A"], p["G"], coarse_size=32)
    oc, gc = O.complexities(H)
    assert len(H) == g["levels"]
    assert oc == pytest.approx(g["oc"], rel=1e-12)
    assert gc == pytest.approx(g["gc"], rel=1e-12)


def test_coarse_gradient_columns_nonzero_and_incidence():
    p = W.hex_problem(6, W.fields.log_uniform(6, 5), 0.01)
    cz = O.coarsen(p["A"], p["G"])
    RG = (cz["R"] @ p["G"]).toarray()
    nzcols = np.flatnonzero(np.abs(RG).sum(axis=0) > 0)
    np.testing.assert_array_equal(cz["coarse_nodes"], nzcols)
    np.testing.assert_array_equal(cz["Gc"].toarray(), RG[:, nzcols])


def test_classical_strength_needed_in_3d_but_not_2d():
    """Reading R3: the symbolic nodal graph stalls 3-D coarse levels; in 2-D both agree."""
    p = W.hex_problem(16, 1.0, 1.0)
    sym = O.setup(p["A"], p["G"], coarse_size=100, strength="symbolic")
    cla = O.setup(p["A"], p["G"], coarse_size=100)
    assert [L["A"].shape[0] for L in cla] == [10800, 1176, 108, 6]
    assert len(sym) == 2
    q = W.tri_problem(16, 1.0, 0.01)
    a = O.setup(q["A"], q["G"], coarse_size=32, strength="symbolic")
    b = O.setup(q["A"], q["G"], coarse_size=32)
    assert [L["A"].nnz for L in a] == [L["A"].nnz for L in b]
