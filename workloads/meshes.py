"""Lowest-order Nedelec (edge element) discretisations of curl(alpha curl u) + beta u = f with u x n = 0.

This is the model problem of the paper (Section 2, Eq. curl): the SPD system A u = f with
A = A^s(alpha) + beta A^m, the curl-curl stiffness A^s and edge mass A^m, and the discrete gradient G
(signed edge/node incidence, de Rham: A^s G = 0).  These generators only build inputs; they hold none
of the multigrid method's arithmetic.

Conventions (shared by every consumer of these inputs):

* Degrees of freedom are line integrals of the tangential field along oriented edges, so G has
  entries -1 (tail) and +1 (head) and a nodal hat's gradient has coefficients G(:, node).
* Boundary edges (lying in the boundary) are eliminated; only interior nodes are columns of G,
  so an interior edge touching the boundary has one nonzero in its G row.
* 3-D hex mesh of the unit cube, n^3 cubes: node (i, j, k), i, j, k in 0..n.  Edges are numbered
  x-edges, then y-edges, then z-edges, each lexicographic (i fastest) by start node and oriented
  along +axis.  Interior nodes (1..n-1)^3 are numbered lexicographically.  DoFs: 3 n (n-1)^2.
* Element matrices by 2x2x2 (3-D) / 2x2 (2-D) Gauss quadrature on the reference cell, which is
  exact for these polynomial integrands.
* 2-D triangle mesh: N x N squares of the unit square, each cut along its (i,j)->(i+1,j+1)
  diagonal; Whitney elements; edges numbered horizontal, vertical, diagonal (DoFs 3N^2 - 2N).
* 2-D quad mesh: N x N squares; edges numbered x-edges then y-edges.
"""
import numpy as np
import scipy.sparse as sp

_GAUSS = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))


def _hat(t, side):
    return t if side else 1.0 - t


def _dhat(side):
    return 1.0 if side else -1.0


# ----------------------------------------------------------------------------------------------
# 3-D hexahedra
# ----------------------------------------------------------------------------------------------
# local edge l: (direction, offset of its start node from the element's origin node)
HEX_LOCAL_EDGES = (
    [(0, (0, b, c)) for (b, c) in ((0, 0), (1, 0), (0, 1), (1, 1))]
    + [(1, (a, 0, c)) for (a, c) in ((0, 0), (1, 0), (0, 1), (1, 1))]
    + [(2, (a, b, 0)) for (a, b) in ((0, 0), (1, 0), (0, 1), (1, 1))]
)


def _hex_basis(l, x, y, z):
    """Reference basis function and its curl at (x, y, z) in [0,1]^3 (unit line integral)."""
    d, (a, b, c) = HEX_LOCAL_EDGES[l]
    if d == 0:
        f = _hat(y, b) * _hat(z, c)
        phi = np.array([f, 0.0, 0.0])
        curl = np.array([0.0, _hat(y, b) * _dhat(c), -_dhat(b) * _hat(z, c)])
    elif d == 1:
        g = _hat(x, a) * _hat(z, c)
        phi = np.array([0.0, g, 0.0])
        curl = np.array([-_hat(x, a) * _dhat(c), 0.0, _dhat(a) * _hat(z, c)])
    else:
        hh = _hat(x, a) * _hat(y, b)
        phi = np.array([0.0, 0.0, hh])
        curl = np.array([_hat(x, a) * _dhat(b), -_dhat(a) * _hat(y, b), 0.0])
    return phi, curl


def hex_element_matrices():
    """Reference 12x12 curl-curl K_ref and mass M_ref on the unit cube (2x2x2 Gauss)."""
    K = np.zeros((12, 12))
    M = np.zeros((12, 12))
    for x in _GAUSS:
        for y in _GAUSS:
            for z in _GAUSS:
                ev = [_hex_basis(l, x, y, z) for l in range(12)]
                for p in range(12):
                    for q in range(12):
                        K[p, q] += 0.125 * ev[p][1] @ ev[q][1]
                        M[p, q] += 0.125 * ev[p][0] @ ev[q][0]
    return K, M


def hex_edge_index(n):
    """Return a function (direction, i, j, k arrays) -> interior edge id, -1 for boundary edges."""
    nm = n - 1
    nx = n * nm * nm

    def eid(d, i, j, k):
        i = np.asarray(i)
        j = np.asarray(j)
        k = np.asarray(k)
        if d == 0:
            ok = (j >= 1) & (j <= nm) & (k >= 1) & (k <= nm) & (i >= 0) & (i < n)
            idx = i + n * ((j - 1) + nm * (k - 1))
        elif d == 1:
            ok = (i >= 1) & (i <= nm) & (k >= 1) & (k <= nm) & (j >= 0) & (j < n)
            idx = nx + (i - 1) + nm * (j + n * (k - 1))
        else:
            ok = (i >= 1) & (i <= nm) & (j >= 1) & (j <= nm) & (k >= 0) & (k < n)
            idx = 2 * nx + (i - 1) + nm * ((j - 1) + nm * k)
        return np.where(ok, idx, -1)

    return eid


def hex_node_index(n):
    nm = n - 1

    def nid(i, j, k):
        i = np.asarray(i)
        j = np.asarray(j)
        k = np.asarray(k)
        ok = (i >= 1) & (i <= nm) & (j >= 1) & (j <= nm) & (k >= 1) & (k <= nm)
        return np.where(ok, (i - 1) + nm * ((j - 1) + nm * (k - 1)), -1)

    return nid


def _assemble(ndof, elem_dofs, Kloc, Mloc, alpha, beta, parts=True):
    """Sum alpha_e K_e + beta_e M_e over elements into sorted CSR; -1 dofs are eliminated.

    Kloc/Mloc: (nl, nl) shared or (ne, nl, nl) per element.  With parts=False the curl-curl and
    mass parts are not assembled separately (returned as None)."""
    ne, nl = elem_dofs.shape
    rows = np.repeat(elem_dofs, nl, axis=1).ravel()
    cols = np.tile(elem_dofs, (1, nl)).ravel()
    if Kloc.ndim == 2:
        kv = (alpha[:, None] * Kloc.ravel()[None, :]).ravel()
        mv = (beta[:, None] * Mloc.ravel()[None, :]).ravel()
    else:
        kv = (alpha[:, None] * Kloc.reshape(ne, -1)).ravel()
        mv = (beta[:, None] * Mloc.reshape(ne, -1)).ravel()
    keep = (rows >= 0) & (cols >= 0)
    rows, cols = rows[keep], cols[keep]
    As = Am = None
    if parts:
        As = sp.coo_matrix((kv[keep], (rows, cols)), shape=(ndof, ndof)).tocsr()
        Am = sp.coo_matrix((mv[keep], (rows, cols)), shape=(ndof, ndof)).tocsr()
        As.sum_duplicates()
        Am.sum_duplicates()
    # same pattern for A, A^s, A^m: assemble the sum directly
    A = sp.coo_matrix((kv[keep] + mv[keep], (rows, cols)), shape=(ndof, ndof)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A, As, Am


def _gradient(ndof, tail, head, nnodes):
    """Signed incidence: -1 at an interior tail node, +1 at an interior head node (-1 = boundary)."""
    r = np.arange(ndof)
    rows = np.concatenate([r[tail >= 0], r[head >= 0]])
    cols = np.concatenate([tail[tail >= 0], head[head >= 0]])
    vals = np.concatenate([-np.ones(int((tail >= 0).sum())), np.ones(int((head >= 0).sum()))])
    G = sp.coo_matrix((vals, (rows, cols)), shape=(ndof, nnodes)).tocsr()
    G.sort_indices()
    return G


def hex_problem(n, alpha, beta, with_parts=False):
    """Assemble A = A^s(alpha) + beta A^m and G on the n^3 hex mesh of the unit cube.

    alpha, beta: scalars or per-element arrays of length n^3 (element (i,j,k) -> i + n(j + n k)).
    Returns dict(A, G, n, ndof, nnodes[, As, Am]) with A, G scipy CSR (sorted, float64)."""
    h = 1.0 / n
    ne = n ** 3
    alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float64), (ne,)).copy()
    beta = np.broadcast_to(np.asarray(beta, dtype=np.float64), (ne,)).copy()
    Kr, Mr = hex_element_matrices()
    K = Kr / h
    M = Mr * h
    eid = hex_edge_index(n)
    e = np.arange(ne)
    ei, ej, ek = e % n, (e // n) % n, e // (n * n)
    elem_dofs = np.empty((ne, 12), dtype=np.int64)
    for l, (d, (a, b, c)) in enumerate(HEX_LOCAL_EDGES):
        elem_dofs[:, l] = eid(d, ei + a, ej + b, ek + c)
    ndof = 3 * n * (n - 1) ** 2
    A, As, Am = _assemble(ndof, elem_dofs, K, M, alpha, beta, parts=with_parts)
    # gradient
    nid = hex_node_index(n)
    tail = np.empty(ndof, dtype=np.int64)
    head = np.empty(ndof, dtype=np.int64)
    nm = n - 1
    for d in range(3):
        if d == 0:
            i, j, k = np.meshgrid(np.arange(n), np.arange(1, n), np.arange(1, n), indexing="ij")
        elif d == 1:
            i, j, k = np.meshgrid(np.arange(1, n), np.arange(n), np.arange(1, n), indexing="ij")
        else:
            i, j, k = np.meshgrid(np.arange(1, n), np.arange(1, n), np.arange(n), indexing="ij")
        i, j, k = i.ravel(), j.ravel(), k.ravel()
        ids = eid(d, i, j, k)
        step = [(1, 0, 0), (0, 1, 0), (0, 0, 1)][d]
        tail[ids] = nid(i, j, k)
        head[ids] = nid(i + step[0], j + step[1], k + step[2])
    G = _gradient(ndof, tail, head, nm ** 3)
    out = dict(A=A, G=G, n=n, ndof=ndof, nnodes=nm ** 3, alpha=alpha, beta=beta, dim=3)
    if with_parts:
        out.update(As=As, Am=Am)
    return out


# ----------------------------------------------------------------------------------------------
# 2-D quadrilaterals
# ----------------------------------------------------------------------------------------------
QUAD_LOCAL_EDGES = [(0, (0, 0)), (0, (0, 1)), (1, (0, 0)), (1, (1, 0))]


def quad_element_matrices():
    K = np.zeros((4, 4))
    M = np.zeros((4, 4))
    for x in _GAUSS:
        for y in _GAUSS:
            phis, curls = [], []
            for d, (a, b) in QUAD_LOCAL_EDGES:
                if d == 0:
                    phis.append(np.array([_hat(y, b), 0.0]))
                    curls.append(-_dhat(b))           # curl = d/dx phi_y - d/dy phi_x
                else:
                    phis.append(np.array([0.0, _hat(x, a)]))
                    curls.append(_dhat(a))
            for p in range(4):
                for q in range(4):
                    K[p, q] += 0.25 * curls[p] * curls[q]
                    M[p, q] += 0.25 * phis[p] @ phis[q]
    return K, M


def quad_problem(N, alpha, beta, with_parts=False):
    """N x N squares of the unit square; x-edges then y-edges, lexicographic by start node."""
    h = 1.0 / N
    ne = N * N
    alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float64), (ne,)).copy()
    beta = np.broadcast_to(np.asarray(beta, dtype=np.float64), (ne,)).copy()
    Kr, Mr = quad_element_matrices()
    K = Kr / h ** 2
    M = Mr
    Nm = N - 1
    nx = N * Nm

    def eid(d, i, j):
        i = np.asarray(i)
        j = np.asarray(j)
        if d == 0:
            ok = (j >= 1) & (j <= Nm) & (i >= 0) & (i < N)
            return np.where(ok, i + N * (j - 1), -1)
        ok = (i >= 1) & (i <= Nm) & (j >= 0) & (j < N)
        return np.where(ok, nx + (i - 1) + Nm * j, -1)

    def nid(i, j):
        ok = (i >= 1) & (i <= Nm) & (j >= 1) & (j <= Nm)
        return np.where(ok, (i - 1) + Nm * (j - 1), -1)

    e = np.arange(ne)
    ei, ej = e % N, e // N
    elem_dofs = np.empty((ne, 4), dtype=np.int64)
    for l, (d, (a, b)) in enumerate(QUAD_LOCAL_EDGES):
        elem_dofs[:, l] = eid(d, ei + a, ej + b)
    ndof = 2 * N * Nm
    A, As, Am = _assemble(ndof, elem_dofs, K, M, alpha, beta)
    tail = np.empty(ndof, dtype=np.int64)
    head = np.empty(ndof, dtype=np.int64)
    i, j = np.meshgrid(np.arange(N), np.arange(1, N), indexing="ij")
    i, j = i.ravel(), j.ravel()
    ids = eid(0, i, j)
    tail[ids], head[ids] = nid(i, j), nid(i + 1, j)
    i, j = np.meshgrid(np.arange(1, N), np.arange(N), indexing="ij")
    i, j = i.ravel(), j.ravel()
    ids = eid(1, i, j)
    tail[ids], head[ids] = nid(i, j), nid(i, j + 1)
    G = _gradient(ndof, tail, head, Nm * Nm)
    out = dict(A=A, G=G, n=N, ndof=ndof, nnodes=Nm * Nm, alpha=alpha, beta=beta, dim=2)
    if with_parts:
        out.update(As=As, Am=Am)
    return out


# ----------------------------------------------------------------------------------------------
# 2-D triangles (Whitney elements)
# ----------------------------------------------------------------------------------------------
def _whitney_triangle(p):
    """Curl-curl and mass matrices of the 3 Whitney functions of triangle p (3x2, CCW).

    Local edge m joins local vertices (a, b) = (0,1), (1,2), (0,2), oriented a -> b:
    phi = lam_a grad lam_b - lam_b grad lam_a, curl phi = 2 grad lam_a x grad lam_b."""
    T = np.array([[1.0, p[0, 0], p[0, 1]], [1.0, p[1, 0], p[1, 1]], [1.0, p[2, 0], p[2, 1]]])
    area = 0.5 * abs(np.linalg.det(T))
    coef = np.linalg.inv(T)               # lam_v(x, y) = coef[0, v] + coef[1, v] x + coef[2, v] y
    grad = coef[1:, :].T                  # grad[v] = (d lam_v/dx, d lam_v/dy)
    pairs = [(0, 1), (1, 2), (0, 2)]
    mm = lambda u, v: area * (2.0 if u == v else 1.0) / 12.0   # integral of lam_u lam_v
    cross = lambda u, v: grad[u][0] * grad[v][1] - grad[u][1] * grad[v][0]
    K = np.zeros((3, 3))
    M = np.zeros((3, 3))
    for r, (a, b) in enumerate(pairs):
        for s, (c, d) in enumerate(pairs):
            K[r, s] = area * 4.0 * cross(a, b) * cross(c, d)
            M[r, s] = (mm(a, c) * grad[b] @ grad[d] - mm(a, d) * grad[b] @ grad[c]
                       - mm(b, c) * grad[a] @ grad[d] + mm(b, d) * grad[a] @ grad[c])
    return K, M


def tri_problem(N, alpha, beta, with_parts=False):
    """N x N squares, each cut along (i,j)->(i+1,j+1).  Element 2(i + N j) is the lower-right
    triangle (i,j),(i+1,j),(i+1,j+1); 2(i + N j) + 1 the upper-left (i,j),(i+1,j+1),(i,j+1)."""
    h = 1.0 / N
    ne = 2 * N * N
    alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float64), (ne,)).copy()
    beta = np.broadcast_to(np.asarray(beta, dtype=np.float64), (ne,)).copy()
    Nm = N - 1
    nh = N * Nm
    nv = Nm * N

    def eid(d, i, j):
        i = np.asarray(i)
        j = np.asarray(j)
        if d == 0:   # horizontal (i,j)->(i+1,j)
            ok = (j >= 1) & (j <= Nm) & (i >= 0) & (i < N)
            return np.where(ok, i + N * (j - 1), -1)
        if d == 1:   # vertical (i,j)->(i,j+1)
            ok = (i >= 1) & (i <= Nm) & (j >= 0) & (j < N)
            return np.where(ok, nh + (i - 1) + Nm * j, -1)
        ok = (i >= 0) & (i < N) & (j >= 0) & (j < N)  # diagonal (i,j)->(i+1,j+1)
        return np.where(ok, nh + nv + i + N * j, -1)

    def nid(i, j):
        ok = (i >= 1) & (i <= Nm) & (j >= 1) & (j <= Nm)
        return np.where(ok, (i - 1) + Nm * (j - 1), -1)

    lower = np.array([[0.0, 0.0], [h, 0.0], [h, h]])
    upper = np.array([[0.0, 0.0], [h, h], [0.0, h]])
    Kl, Ml = _whitney_triangle(lower)
    Ku, Mu = _whitney_triangle(upper)
    s = np.arange(N * N)
    si, sj = s % N, s // N
    # lower: local edges (0,1) horizontal (+), (1,2) vertical at i+1 (+), (0,2) diagonal (+)
    dl = np.stack([eid(0, si, sj), eid(1, si + 1, sj), eid(2, si, sj)], axis=1)
    # upper: local edges (0,1) diagonal (+), (1,2) horizontal at j+1 reversed, (0,2) vertical at i (+)
    du = np.stack([eid(2, si, sj), eid(0, si, sj + 1), eid(1, si, sj)], axis=1)
    su = np.array([1.0, -1.0, 1.0])
    Ku = Ku * np.outer(su, su)
    Mu = Mu * np.outer(su, su)
    elem_dofs = np.empty((ne, 3), dtype=np.int64)
    elem_dofs[0::2] = dl
    elem_dofs[1::2] = du
    Kloc = np.empty((ne, 3, 3))
    Mloc = np.empty((ne, 3, 3))
    Kloc[0::2], Kloc[1::2] = Kl, Ku
    Mloc[0::2], Mloc[1::2] = Ml, Mu
    ndof = 3 * N * N - 2 * N
    A, As, Am = _assemble(ndof, elem_dofs, Kloc, Mloc, alpha, beta)
    tail = np.empty(ndof, dtype=np.int64)
    head = np.empty(ndof, dtype=np.int64)
    for d, (di, dj), irange, jrange in ((0, (1, 0), range(N), range(1, N)),
                                         (1, (0, 1), range(1, N), range(N)),
                                         (2, (1, 1), range(N), range(N))):
        i, j = np.meshgrid(np.array(list(irange)), np.array(list(jrange)), indexing="ij")
        i, j = i.ravel(), j.ravel()
        ids = eid(d, i, j)
        tail[ids], head[ids] = nid(i, j), nid(i + di, j + dj)
    G = _gradient(ndof, tail, head, Nm * Nm)
    out = dict(A=A, G=G, n=N, ndof=ndof, nnodes=Nm * Nm, alpha=alpha, beta=beta, dim=2)
    if with_parts:
        out.update(As=As, Am=Am)
    return out
