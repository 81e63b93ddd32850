"""Pins of two oracle parts that only 3-D or mixed-precision runs reach: the ring-neighbourhood
branch of the local patches (Eq. sparseP with reading R1, the branch every 3-D patch takes) and
flexible CG (Section 5's solver with a preconditioner that is not a fixed SPD operator)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import amg as O


# ---------------------------------------------------------------------------------------------
# ring-neighbourhood patches
# ---------------------------------------------------------------------------------------------
def brute_force_ring_patch(adj, ext, d1, d2, ring, p_max):
    """Ring patch of the exterior pair (d1, d2) from a dense distance table: an interior DoF's
    distance is the least number of steps through A's pattern from {d1, d2} with every
    intermediate DoF interior.  Keep distances 1..ring, order by (distance, index), keep the first
    p_max, return them ascending."""
    n = adj.shape[0]
    dist = np.full(n, np.inf)
    frontier = np.zeros(n, bool)
    frontier[[d1, d2]] = True
    reached = frontier.copy()
    for step in range(1, ring + 1):
        nxt = (adj[frontier].any(axis=0)) & ~ext & ~reached
        dist[nxt] = step
        reached |= nxt
        frontier = nxt
    cand = np.flatnonzero(np.isfinite(dist))
    order = sorted(cand.tolist(), key=lambda d: (dist[d], d))
    return np.array(sorted(order[:p_max]), dtype=np.int64)


def _ext_mask(edges, n):
    ext = np.zeros(n, bool)
    for e in edges:
        ext[e[0]] = ext[e[2]] = True
    return ext


@pytest.mark.parametrize("n,ring,p_max", [(4, 1, 4), (5, 1, 20), (6, 2, 128), (7, 2, 100),
                                          (7, 3, 200)])
def test_ring_patches_match_brute_force(n, ring, p_max):
    """R1's second branch on 3-D hexes: where the touched components of graph(A_II) exceed p_max
    the patch is the ring-`ring` interior neighbourhood of the pair, truncated in BFS order with
    ties by index.  Every patch is checked against a dense distance table; exterior DoFs never
    enter a patch."""
    p = W.hex_problem(n, W.fields.log_uniform(n, 5, lo=-1.0, hi=1.0), 0.1)
    A = sp.csr_matrix(p["A"])
    cz = O.coarsen(A, p["G"])
    edges = cz["edges"]
    ndof = A.shape[0]
    ext = _ext_mask(edges, ndof)
    adj = (A.toarray() != 0)
    np.fill_diagonal(adj, False)
    patches = O.interior_patches(A, edges, ndof, p_max=p_max, ring=ring)
    n_interior = int((~ext).sum())
    truncated = 0
    for e, patch in zip(edges, patches):
        assert not ext[patch].any()
        want = brute_force_ring_patch(adj, ext, e[0], e[2], ring, p_max)
        if p_max >= n_interior:
            continue            # the component branch may take the whole interior instead
        np.testing.assert_array_equal(patch, want)
        truncated += len(want) == p_max
    assert truncated > 0        # every case truncates some patch inside its last ring


def test_3d_interior_graph_is_one_component_and_ring_branch_taken():
    """In 3-D the exterior skeleton does not separate graph(A_II), so with the default p_max
    every hex patch comes from the ring branch: it holds only distance-1 interior DoFs."""
    n = 6
    p = W.hex_problem(n, 1.0, 1.0)
    A = sp.csr_matrix(p["A"])
    cz = O.coarsen(A, p["G"])
    ext = _ext_mask(cz["edges"], A.shape[0])
    adj = (A.toarray() != 0)
    np.fill_diagonal(adj, False)
    I = np.flatnonzero(~ext)
    # one component: a breadth-first closure from the first interior DoF reaches all of them
    seen = np.zeros(A.shape[0], bool)
    seen[I[0]] = True
    while True:
        grow = adj[seen].any(axis=0) & ~ext & ~seen
        if not grow.any():
            break
        seen |= grow
    assert seen[I].all() and len(I) > 128
    for e, patch in zip(cz["edges"], cz["patches"]):
        np.testing.assert_array_equal(patch, brute_force_ring_patch(adj, ext, e[0], e[2], 1, 128))


def test_patches_covering_the_interior_give_the_global_interpolation():
    """With p_max >= |I| on a 3-D hex, every patch is the whole (connected) interior, so the local
    solves are the exact interior solve of Eq. sparseP and P equals the global P_app."""
    n = 4
    p = W.hex_problem(n, W.fields.log_uniform(n, 6, lo=-0.5, hi=0.5), 1.0)
    A = sp.csr_matrix(p["A"])
    loc = O.coarsen(A, p["G"], p_max=10 ** 6)
    glo = O.coarsen(A, p["G"], interp="global")
    ext = _ext_mask(loc["edges"], A.shape[0])
    I = np.flatnonzero(~ext)
    for patch in loc["patches"]:
        np.testing.assert_array_equal(patch, I)
    np.testing.assert_allclose(loc["P"].toarray(), glo["P"].toarray(), atol=1e-11, rtol=0)


# ---------------------------------------------------------------------------------------------
# flexible CG
# ---------------------------------------------------------------------------------------------
def _iterates(H, f, flexible, precond_factory, k_max):
    """x_k for k = 1..k_max: separate runs stopped after k iterations (every run starts a fresh
    preconditioner sequence, so run k reproduces the first k steps of run k_max)."""
    return [O.pcg(H, f, tol=0.0, maxit=k, flexible=flexible, precond=precond_factory())[0]
            for k in range(1, k_max + 1)]


def _small_hierarchy():
    p = W.hex_problem(6, W.fields.checkerboard(6, 3, hi=1e2), 0.1)
    H = O.setup(p["A"], p["G"], coarse_size=60)
    return p, H, W.fields.rhs(p["ndof"], 0)


def test_flexible_cg_reproduces_pcg_with_a_fixed_spd_preconditioner():
    """With a fixed symmetric positive definite preconditioner, z_k+1 is orthogonal to r_k, so the
    flexible (Polak-Ribiere) beta equals the Fletcher-Reeves one and the iterates coincide."""
    p, H, f = _small_hierarchy()
    A = p["A"]
    fixed = lambda: (lambda r: O.vcycle(H, r))
    xs_p = _iterates(H, f, False, fixed, 8)
    xs_f = _iterates(H, f, True, fixed, 8)
    for k, (a, b) in enumerate(zip(xs_p, xs_f), 1):
        d = a - b
        err = np.sqrt(d @ (A @ d) / (a @ (A @ a)))
        assert err < 1e-10, (k, err)


def test_flexible_cg_keeps_consecutive_directions_conjugate_with_a_varying_preconditioner():
    """Flexible CG's beta makes each new direction A-conjugate to the previous one whatever the
    preconditioner does.  With a preconditioner that alternates between the V-cycle and
    l1-Jacobi, the steps d_k = x_k+1 - x_k of flexible CG stay pairwise conjugate; those of the
    Fletcher-Reeves recurrence do not (which shows the check can tell the two apart)."""
    p, H, f = _small_hierarchy()
    A = p["A"]
    l1 = O.l1_diagonal(A)

    def alternating():
        state = {"k": 0}

        def B(r):
            state["k"] += 1
            return O.vcycle(H, r) if state["k"] % 2 else r / l1
        return B

    def max_cos(flexible):
        xs = [np.zeros_like(f)] + _iterates(H, f, flexible, alternating, 7)
        ds = [xs[k + 1] - xs[k] for k in range(len(xs) - 1)]
        an = lambda u: np.sqrt(u @ (A @ u))
        return max(abs(ds[k + 1] @ (A @ ds[k])) / (an(ds[k + 1]) * an(ds[k]))
                   for k in range(len(ds) - 1))

    assert max_cos(True) < 1e-9
    assert max_cos(False) > 1e-4
