"""Pins of the refinement-based coarse variables ("Ref", Sec. 3) and the geometric Nedelec
interpolation ("Geo", the comparison of Sec. 5) on the structured hex mesh: the coarse gradient
is the coarse mesh's own, the geometric interpolation commutes with the gradient and trilinear
nodal interpolation exactly, and on an isotropic mesh the algebraic splitting (Alg. 2-3) finds the
same coarse edges as the refinement, so both build the same interpolation."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import amg as O


def trilinear_nodal_interpolation(n):
    """Interior nodes of the (n/2)^3 mesh -> interior nodes of the n^3 mesh by trilinear
    interpolation (boundary nodes carry zero), written from the node coordinates."""
    N = n // 2
    m, M = n - 1, N - 1
    rows, cols, vals = [], [], []
    for z in range(1, n):
        for y in range(1, n):
            for x in range(1, n):
                r = (x - 1) + m * ((y - 1) + m * (z - 1))
                for X in (x // 2, (x + 1) // 2) if x % 2 else (x // 2,):
                    for Y in (y // 2, (y + 1) // 2) if y % 2 else (y // 2,):
                        for Z in (z // 2, (z + 1) // 2) if z % 2 else (z // 2,):
                            if 1 <= X <= M and 1 <= Y <= M and 1 <= Z <= M:
                                w = (0.5 if x % 2 else 1.0) * (0.5 if y % 2 else 1.0) * (0.5 if z % 2 else 1.0)
                                rows.append(r)
                                cols.append((X - 1) + M * ((Y - 1) + M * (Z - 1)))
                                vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(m ** 3, max(M, 0) ** 3))


@pytest.mark.parametrize("n", [4, 8, 12])
def test_refinement_coarse_gradient_is_the_coarse_mesh_gradient(n):
    """Eq. Gc with the refinement pairs: R G keeps exactly the interior coarse nodes, in their
    order, and equals the (n/2)^3 mesh's signed incidence (every row e_head - e_tail)."""
    p = W.hex_problem(n, 1.0, 1.0)
    edges = O.refinement_edges(n)
    R = O.restriction(edges, p["ndof"])
    Gc, keep = O.coarse_gradient(p["G"], R)
    pc = W.hex_problem(n // 2, 1.0, 1.0)
    assert Gc.shape == pc["G"].shape
    assert abs(Gc - pc["G"]).max() == 0
    # the halves are distinct fine DoFs, oriented like their coarse edge (R rows (+1, +1))
    d = np.array([[e[0], e[2]] for e in edges])
    assert len(np.unique(d)) == d.size
    assert all(e[1] == 1.0 and e[3] == 1.0 for e in edges)


@pytest.mark.parametrize("n", [4, 6, 8])
def test_geometric_interpolation_commutes(n):
    """Geo P G_c = 2 G P_n with P_n the trilinear nodal interpolation (the commuting diagram of
    lowest-order Nedelec and trilinear Lagrange elements), exactly; its rows on each coarse edge's
    two halves are R^T."""
    p = W.hex_problem(n, 1.0, 1.0)
    edges = O.refinement_edges(n)
    P = O.interpolation_geometric(n, edges, p["ndof"])
    Gc = W.hex_problem(n // 2, 1.0, 1.0)["G"]
    Pn = trilinear_nodal_interpolation(n)
    assert abs(P @ Gc - 2.0 * (p["G"] @ Pn)).max() == 0
    R = O.restriction(edges, p["ndof"])
    ext = np.concatenate([[e[0], e[2]] for e in edges])
    np.testing.assert_array_equal(P[ext].toarray(), R.T.tocsr()[ext].toarray())
    # a column inside the mesh holds its two halves and 16 parallel neighbours
    counts = np.diff(P.tocsc().indptr)
    assert counts.max() == 18


def test_geometric_interpolation_reproduces_a_nodal_gradient_field():
    """A smooth discrete gradient on the coarse mesh interpolates to the gradient of the
    trilinear interpolant on the fine mesh (the commuting property applied to one field)."""
    n = 8
    p = W.hex_problem(n, 1.0, 1.0)
    edges = O.refinement_edges(n)
    P = O.interpolation_geometric(n, edges, p["ndof"])
    phi = W.uniform("probe", 11, (n // 2 - 1) ** 3)
    Gc = W.hex_problem(n // 2, 1.0, 1.0)["G"]
    np.testing.assert_allclose(P @ (Gc @ phi), 2.0 * (p["G"] @ (trilinear_nodal_interpolation(n) @ phi)),
                               rtol=0, atol=1e-14)


def test_algebraic_splitting_equals_refinement_on_an_isotropic_mesh():
    """On the uniform isotropic 8^3 hex mesh Alg. 2-3 pair the same fine DoFs as the geometric
    refinement (each coarse edge's two halves), so the local harmonic extensions (Eq. sparseP)
    give the same columns up to order and sign."""
    n = 8
    p = W.hex_problem(n, 1.0, 1.0)
    alg = O.coarsen(p["A"], p["G"])
    ref = O.coarsen(p["A"], p["G"], splitting="refinement", mesh_n=n)
    pa = {frozenset((e[0], e[2])): c for c, e in enumerate(alg["edges"])}
    pr = {frozenset((e[0], e[2])): c for c, e in enumerate(ref["edges"])}
    assert set(pa) == set(pr)
    Pa, Pr = alg["P"].tocsc(), ref["P"].tocsc()
    for key, ca in pa.items():
        a = Pa[:, ca].toarray().ravel()
        r = Pr[:, pr[key]].toarray().ravel()
        sign = 1.0 if a @ r >= 0 else -1.0
        np.testing.assert_allclose(a, sign * r, rtol=0, atol=1e-13)


def test_refinement_hierarchy_levels():
    """The refinement hierarchy halves the mesh per level (DoFs 3 n (n-1)^2) while it stays even."""
    p = W.hex_problem(16, W.fields.checkerboard(16, 4), 1e-2)
    H = O.setup(p["A"], p["G"], splitting="refinement", mesh_n=16, coarse_size=100)
    assert [L["A"].shape[0] for L in H] == [10800, 1176, 108, 6]
    Hg = O.setup(p["A"], p["G"], splitting="refinement", mesh_n=16, coarse_size=100, interp="geometric")
    assert [L["A"].shape[0] for L in Hg] == [10800, 1176, 108, 6]
    f = W.fields.rhs(p["ndof"], 0)
    _, it_ref, _ = O.pcg(H, f, tol=1e-8)
    _, it_geo, _ = O.pcg(Hg, f, tol=1e-8)
    print("16^3 checkerboard PCG iterations: Ref %d, Geo %d" % (it_ref, it_geo))
    assert it_ref < 200 and it_geo < 500
