"""Pins of the oracle's commuting correction of the local extension (interp="constrained"; Eq.
commuting with Eq. sparseP, readings R10-R11): the nodal interpolation is trilinear on a hex
refinement, the exterior rows R^T satisfy P G_c = 2 G P_n before any correction, every corrected
row is the nearest one on its pattern (checked against the KKT system of that least-distance
problem, solved another way), the corrected P commutes, and in 3-D it converges faster than the
plain local extension."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import amg as O
from test_oracle_refinement import trilinear_nodal_interpolation


def defect(cz, G):
    m = G.shape[1]
    return sp.csr_matrix(cz["P"] @ cz["Gc"] - 2.0 * (sp.csr_matrix(G) @ cz["Pn"][:m]))


def exterior(cz, n):
    ext = np.zeros(n, dtype=bool)
    for e in cz["edges"]:
        ext[e[0]] = ext[e[2]] = True
    return ext


@pytest.mark.parametrize("n", [4, 6, 8])
def test_nodal_interpolation_is_trilinear_on_a_hex_refinement(n):
    """R10 on the refinement pairs of the n^3 mesh: coarse nodes injected, edge midpoints, face and
    cell centres averaged layer by layer, boundary nodes zero -> trilinear interpolation."""
    p = W.hex_problem(n, 1.0, 1.0)
    cz = O.coarsen(p["A"], p["G"], splitting="refinement", mesh_n=n, interp="constrained")
    m = p["G"].shape[1]
    np.testing.assert_allclose(cz["Pn"][:m].toarray(), trilinear_nodal_interpolation(n).toarray(), rtol=0, atol=1e-15)
    # the artificial boundary columns of G~ are zero rows
    assert abs(cz["Pn"][m:]).max() == 0 if cz["Pn"].shape[0] > m else True


CASES = {
    "hex8_unit": lambda: W.make_config("hex8_unit"),
    "hex12_lognormal": lambda: W.hex_problem(12, W.fields.log_uniform(12, 3, lo=-2, hi=2), 0.1),
    "tri16": lambda: W.tri_problem(16, 1.0, 0.01),
}


@pytest.fixture(scope="module", params=list(CASES))
def pair(request):
    p = CASES[request.param]()
    A, G = p["A"], p["G"]
    loc = O.coarsen(A, G)
    con = O.coarsen(A, G, interp="constrained")
    return request.param, A, G, loc, con


def test_exterior_rows_commute_before_correction(pair):
    """R^T rows with the middle node's halves: a half edge carries half of its coarse edge's
    difference, so the uncorrected local extension already satisfies the relation on them."""
    name, A, G, loc, con = pair
    d = defect(dict(loc, Pn=con["Pn"]), G)
    ext = exterior(con, A.shape[0])
    assert abs(d[np.flatnonzero(ext)]).max() <= 1e-15, name
    # and not on the interior rows of a 3-D patch extension (otherwise nothing is pinned)
    if name.startswith("hex"):
        assert abs(d[np.flatnonzero(~ext)]).max() > 1e-3


def test_corrected_rows_commute_and_keep_the_pattern(pair):
    name, A, G, loc, con = pair
    Pl, Pc = sp.csr_matrix(loc["P"]), sp.csr_matrix(con["P"])
    np.testing.assert_array_equal(Pl.indptr, Pc.indptr)
    np.testing.assert_array_equal(Pl.indices, Pc.indices)
    ext = np.flatnonzero(exterior(con, A.shape[0]))
    assert abs(Pl[ext] - Pc[ext]).max() == 0
    d = defect(con, G)
    print("%s: max |P G_c - 2 G P_n| = %.2e, max |P_con - P_loc| = %.3f" % (name, abs(d).max(), abs(Pc - Pl).max()))
    assert abs(d).max() <= 1e-13


def test_each_row_is_the_nearest_on_its_pattern(pair):
    """Least distance to the local row under row i of the relation, solved through its KKT system
    [I C; C^T 0] [p; lam] = [p0; t] (consistent, possibly singular: lstsq), on sampled rows."""
    name, A, G, loc, con = pair
    Pl, Pc = sp.csr_matrix(loc["P"]), sp.csr_matrix(con["P"])
    Gc = sp.csr_matrix(con["Gc"])
    T = sp.csr_matrix(2.0 * (sp.csr_matrix(G) @ con["Pn"][:G.shape[1]]))
    inner = np.flatnonzero(~exterior(con, A.shape[0]) & (np.diff(Pl.indptr) > 0))
    rng = np.random.default_rng(5)
    for i in rng.choice(inner, min(60, len(inner)), replace=False):
        S = Pl.indices[Pl.indptr[i]:Pl.indptr[i + 1]]
        C = Gc[S].toarray()
        t = T[i].toarray().ravel()
        k, m = C.shape
        K = np.block([[np.eye(k), C], [C.T, np.zeros((m, m))]])
        sol = np.linalg.lstsq(K, np.concatenate([Pl[i, S].toarray().ravel(), t]), rcond=1e-10)[0]
        assert np.allclose(sol[:k] @ C, t, rtol=0, atol=1e-12), (name, i)
        np.testing.assert_allclose(Pc[i, S].toarray().ravel(), sol[:k], rtol=0, atol=1e-12)


def test_correction_is_idempotent(pair):
    name, A, G, loc, con = pair
    again = O.interpolation_constrained(con["P"], G, con["Gc"], con["Pn"], con["edges"])
    assert abs(again - con["P"]).max() <= 1e-14


def test_a_row_without_a_commuting_choice_is_corrected_in_least_squares():
    """A pattern too small for the relation: the correction leaves the smallest residual (what is
    left is orthogonal to every achievable change) with the smallest change."""
    # one fine row, coarse gradient rows: c0 = e1 - e0, c1 = e2 - e1; pattern {c0}
    Gc = sp.csr_matrix(np.array([[-1.0, 1.0, 0.0], [0.0, -1.0, 1.0]]))
    P = sp.csr_matrix(np.array([[0.3, 0.0], [1.0, 0.0], [0.0, 1.0]]))
    G = sp.csr_matrix(np.array([[-1.0, 1.0], [0.0, 1.0], [1.0, 0.0]]))
    Pn = sp.csr_matrix(np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]]))
    edges = [(1, 1.0, 1, 1.0, 0, -1, 1), (2, 1.0, 2, 1.0, 1, -1, 2)]
    out = O.interpolation_constrained(P, G, Gc, Pn, edges)
    # row 0: t = 2 (Pn[1] - Pn[0]) = (-2, 0, 2); achievable p (-1, 1, 0); least squares
    # p = <(-1, 1, 0), t> / 2 = 1
    assert out[0, 0] == pytest.approx(1.0, abs=1e-14)
    r = out[0, 0] * np.array([-1.0, 1.0, 0.0]) - np.array([-2.0, 0.0, 2.0])
    assert abs(r @ np.array([-1.0, 1.0, 0.0])) < 1e-14
    assert abs(out[1:] - P[1:]).max() == 0


def test_three_dimensional_convergence():
    """The point of the correction: on the 16^3 checkerboard the commuting P takes fewer PCG
    iterations than the plain local extension (15 here), for both coarse-variable choices."""
    p = W.make_config("hex16_checker")
    its = {}
    for label, kw in (("local", {}), ("constrained", dict(interp="constrained")),
                      ("ref constrained", dict(interp="constrained", splitting="refinement", mesh_n=16))):
        H = O.setup(p["A"], p["G"], **kw)
        its[label] = O.pcg(H, p["f"], tol=1e-8)[1]
    print("16^3 checkerboard PCG iterations:", its)
    assert its["constrained"] <= its["local"] - 3
    assert its["ref constrained"] <= its["local"] - 3


def test_rank_of_the_row_block_is_structural():
    """A row whose block C (an incidence block of 27 coarse edges on 27 coarse nodes: one
    ungrounded component plus a node only the target touches, so two exact zero singular values,
    one of which the SVD returns as ~2e-14) met on the 64^3 checkerboard's third level: the
    correction must equal the structural least-squares solution (mean of the residual removed on
    the component, the untouched node dropped, one node pinned, the graph Laplacian solved) and
    stay bounded, where a default pseudo-inverse cutoff keeps the noise and returns 1e13."""
    ends = [(1, 11), (2, 14), (3, 15), (4, 16), (5, 9), (6, 10), (7, 11), (8, 9), (9, 10), (9, 14), (9, 21),
            (10, 11), (10, 15), (10, 22), (11, 12), (11, 16), (11, 23), (13, 14), (14, 15), (14, 18), (14, 24),
            (15, 16), (15, 19), (15, 25), (16, 17), (16, 20), (16, 26)]
    p0 = np.array([0.0667232, 1.55595e-05, 0.374158, 0.125761, 1.87685e-06, 5.10011e-06, 6.86364e-06,
                   -3.27861e-07, -2.50915e-06, 0.00329235, 0.0013778, -0.0103606, -0.00638136, 0.0146981,
                   -1.55354e-06, 0.000105693, 0.0131414, 1.40856e-07, -0.0493808, -0.00309791, -0.00103133,
                   -0.0174202, 0.0164795, 0.0221993, -2.25032e-06, 0.00330395, 0.00683052])
    k, m = len(ends), 27
    C = np.zeros((k, m))
    for e, (u, v) in enumerate(ends):
        C[e, u], C[e, v] = -1.0, 1.0
    Gc = sp.csr_matrix(C)
    # fine row 0 (interior) with all 27 coarse edges in its pattern; fine row 1 holds the pairs
    P = sp.csr_matrix((p0, (np.zeros(k, int), np.arange(k))), shape=(2, k))
    G = sp.csr_matrix(np.array([[-1.0, 1.0], [0.0, 1.0]]))
    Pn = sp.csr_matrix(np.array([[0.25 if c in (0, 3) else 0.0 for c in range(m)],
                                 [0.25 if c in (10, 15) else 0.0 for c in range(m)]]))
    edges = [(1, 1.0, 1, 1.0, -1, -1, -1)]
    t = 2.0 * (G @ Pn).toarray()[0]
    out = O.interpolation_constrained(P, G, Gc, Pn, edges).toarray()[0]
    # structural solution: nodes 1..26 form one ungrounded component, node 0 is untouched
    r = t - p0 @ C
    comp = np.arange(1, m)
    r_c = r[comp] - r[comp].mean()
    act = comp[1:]                        # node 1 pinned
    L = C.T @ C
    y = np.zeros(m)
    y[act] = np.linalg.solve(L[np.ix_(act, act)], r_c[1:])
    want = p0 + C @ y
    assert np.abs(out).max() < 10.0
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-12)


def test_every_level_of_a_hierarchy_commutes():
    """The correction on every level of a corrected hierarchy (coarse levels come from Galerkin
    products of corrected P, so their gradients are the coarse G_c): the relation holds to rounding
    on each level, and each level's exterior rows are R^T."""
    p = W.hex_problem(12, W.fields.log_uniform(12, 3, lo=-2, hi=2), 0.1)
    H = O.setup(p["A"], p["G"], interp="constrained")
    assert len(H) >= 3
    for l, L in enumerate(H[:-1]):
        cz = L["coarsening"]
        G = sp.csr_matrix(L["G"])
        d = defect(cz, G)
        assert abs(d).max() <= 1e-12 * max(1.0, abs(cz["P"]).max()), (l, abs(d).max())
        ext = np.concatenate([[e[0], e[2]] for e in cz["edges"]])
        R = O.restriction(cz["edges"], L["A"].shape[0])
        assert abs(sp.csr_matrix(cz["P"])[ext] - R.T.tocsr()[ext]).max() == 0, l
