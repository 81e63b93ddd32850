"""Pins of the learned-interpolation reference: finite-difference gradients, the closed-form first
Adam step, and translation invariance of the patch features and exact targets on a uniform mesh."""
import numpy as np

import workloads as W
from oracle import amg as O
from oracle import mlp as M


def _u01(seed):
    return lambda count, offset=0: W.uniform01("mlp", seed, count, offset)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    d_in, width, d_out, nb = 7, 5, 4, 6
    params = M.init_params(_u01(1), d_in, width, d_out)
    params = [p + 0.1 * rng.standard_normal(p.shape) for p in params]   # nonzero biases too
    X = rng.standard_normal((nb, d_in))
    T = rng.standard_normal((nb, d_out))
    Mk = (rng.random((nb, d_out)) < 0.7).astype(float)
    L, grads = M.backward(params, X, T, Mk)
    assert abs(L - M.loss(params, X, T, Mk)) < 1e-14
    h = 1e-6
    for pi, p in enumerate(params):
        for idx in np.ndindex(p.shape):
            pp = [q.copy() for q in params]
            pm = [q.copy() for q in params]
            pp[pi][idx] += h
            pm[pi][idx] -= h
            fd = (M.loss(pp, X, T, Mk) - M.loss(pm, X, T, Mk)) / (2 * h)
            assert abs(fd - grads[pi][idx]) < 1e-6 * max(1.0, abs(fd)), (pi, idx)


def test_first_adam_step_is_signed_lr():
    # with bias correction the first step is -lr * g / (|g| + eps)
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -1e-3, 0.0])]
    out = M.adam_step(p, g, [], lr=0.01, t=1)
    np.testing.assert_allclose(out[0], p[0] - 0.01 * g[0] / (np.abs(g[0]) + 1e-8), rtol=1e-14)


def test_zero_network_predicts_bias():
    X = np.ones((3, M.D_IN))
    params = [np.zeros((M.D_IN, 8)), np.zeros(8), np.zeros((8, 8)), np.zeros(8), np.zeros((8, M.M_IN)),
              np.linspace(-1, 1, M.M_IN)]
    y, _ = M.forward(params, X)
    np.testing.assert_array_equal(y, np.tile(params[5], (3, 1)))


def test_features_and_targets_are_translation_invariant():
    """Interior coarse edges of a uniform isotropic mesh that differ by a coarse-grid translation
    have identical local problems: identical features and identical exact targets."""
    n = 12
    p = W.hex_problem(n, 1.0, 0.5)
    cz = O.coarsen(p["A"], p["G"])
    nm = n - 1
    xyz = lambda v: np.array([v % nm + 1, (v // nm) % nm + 1, v // (nm * nm) + 1])
    groups = {}
    for c, e in enumerate(cz["edges"]):
        i, k, j = e[4], e[5], e[6]
        if j >= p["G"].shape[1]:
            continue
        a, b = xyz(i), xyz(j)
        # well inside: the patch sees no boundary
        if a.min() < 4 or b.max() > n - 4:
            continue
        groups.setdefault(tuple(b - a), []).append(c)
    assert groups and all(len(v) >= 2 for v in groups.values())
    for cs in groups.values():
        f0, m0 = M.patch_features(p["A"], cz["edges"][cs[0]], cz["patches"][cs[0]])
        t0 = M.patch_target(p["A"], cz["edges"][cs[0]], cz["patches"][cs[0]])
        assert m0.sum() == len(cz["patches"][cs[0]]) and 0 < m0.sum() <= M.M_IN
        for c in cs[1:]:
            f, m = M.patch_features(p["A"], cz["edges"][c], cz["patches"][c])
            t = M.patch_target(p["A"], cz["edges"][c], cz["patches"][c])
            np.testing.assert_allclose(f, f0, atol=1e-12)
            np.testing.assert_allclose(t, t0, atol=1e-12)
        # the target is the column of P on the patch
        col = cz["P"][:, cs[0]].toarray().ravel()
        np.testing.assert_allclose(t0[:len(cz["patches"][cs[0]])], col[cz["patches"][cs[0]]], atol=1e-13)


def test_learned_interpolation_of_a_zero_network_is_the_restriction():
    """A network with zero weights and biases predicts 0 inside every patch: P = R^T (Eq. sparseP
    with the interior part dropped), and the learned hierarchy is built on it."""
    p = W.hex_problem(6, 1.0, 1.0)
    cz = O.coarsen(p["A"], p["G"])
    params = [np.zeros((M.D_IN, 8)), np.zeros(8), np.zeros((8, 8)), np.zeros(8), np.zeros((8, M.M_IN)),
              np.zeros(M.M_IN)]
    P = M.learned_interpolation(p["A"], cz["edges"], cz["patches"], p["ndof"], params)
    R = O.restriction(cz["edges"], p["ndof"])
    assert abs(P - R.T).max() == 0.0
    H = M.setup_learned(p["A"], p["G"], params)
    assert abs(H[0]["P"] - R.T).max() == 0.0
    np.testing.assert_allclose(H[1]["A"].toarray(), (R @ p["A"] @ R.T).toarray(), rtol=0, atol=1e-13)


def test_learned_interpolation_places_predictions_on_the_patch():
    """A network whose last layer is a bias b3 puts b3[q] at the q-th DoF of every patch."""
    p = W.hex_problem(6, 1.0, 1.0)
    cz = O.coarsen(p["A"], p["G"])
    b3 = np.linspace(0.5, 1.5, M.M_IN)
    params = [np.zeros((M.D_IN, 8)), np.zeros(8), np.zeros((8, 8)), np.zeros(8), np.zeros((8, M.M_IN)), b3]
    P = M.learned_interpolation(p["A"], cz["edges"], cz["patches"], p["ndof"], params).tolil()
    for c, (e, pt) in enumerate(zip(cz["edges"], cz["patches"])):
        assert P[e[0], c] == e[1] and P[e[2], c] == e[3]
        for q, g in enumerate(pt):
            assert P[g, c] == b3[q]
        assert P[:, c].nnz == len(pt) + 2


def test_probe_factor_obeys_the_energy_bound():
    """The symmetric V-cycle's error propagator E = I - B A is A-self-adjoint, so after k cycles
    ||A e_k|| / ||A e_0|| <= sqrt(kappa(A)) rho(E)^k: the probe factor is at most
    rho(E) kappa(A)^(1/2k), and it equals the ratio computed from the dense E."""
    p = W.hex_problem(5, 1.0, 1.0)
    H = O.setup(p["A"], p["G"], coarse_size=100)
    assert len(H) >= 2
    n = p["ndof"]
    A = p["A"].toarray()
    B = np.column_stack([O.vcycle(H, np.eye(n)[:, j]) for j in range(n)])
    E = np.eye(n) - B @ A
    rho = max(abs(np.linalg.eigvals(E)))
    lam = np.linalg.eigvalsh(A)
    x0 = W.uniform("probe", 0, n)
    k = 10
    f = O.probe_factor(H, x0, k)
    assert 0.0 < rho < 1.0
    assert f <= rho * (lam[-1] / lam[0]) ** (0.5 / k) * (1 + 1e-12)
    ek = np.linalg.matrix_power(E, k) @ x0
    assert abs(f - (np.linalg.norm(A @ ek) / np.linalg.norm(A @ x0)) ** (1.0 / k)) < 1e-9


def test_bf16_rounding_is_nearest_even_of_the_float32_value():
    """to_bf16 against hand-placed ties and against torch's own float32 -> bfloat16 conversion
    (round to nearest, ties to even) on random values."""
    torch = __import__("pytest").importorskip("torch")
    u = 2.0 ** -8                      # half a bfloat16 unit at 1 (8 significant bits)
    vals = np.array([1.0, 1 + u, 1 + 3 * u, 1 + u + 2.0 ** -20, -(1 + 3 * u), 3.0, 0.0, 2.0 ** -130])
    want = np.array([1.0, 1.0, 1 + 4 * u, 1 + 2 * u, -(1 + 4 * u), 3.0, 0.0, 2.0 ** -130])
    np.testing.assert_array_equal(M.to_bf16(vals), want)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(20000) * 10.0 ** rng.uniform(-6, 6, 20000)
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.to_bf16(x), ref)


def test_bf16_storage_changes_only_what_it_rounds():
    """With inputs, weights and every hidden activation already bfloat16 values (small integers and
    halves), BF16 storage gives exactly the FP32 forward pass and gradients; with general values
    the forward pass differs, by about the bfloat16 unit."""
    rng = np.random.default_rng(2)
    d_in, width, d_out, nb = 6, 5, 4, 3
    ints = lambda shape: rng.integers(-3, 4, shape).astype(float) / 2.0
    params = [ints((d_in, width)), ints(width), ints((width, width)), ints(width), ints((width, d_out)), ints(d_out)]
    X, T, Mk = ints((nb, d_in)), ints((nb, d_out)), np.ones((nb, d_out))
    y32, _ = M.forward(params, X)
    y16, _ = M.forward(params, X, "bf16")
    np.testing.assert_array_equal(y16, y32)
    L32, g32 = M.backward(params, X, T, Mk)
    L16, g16 = M.backward(params, X, T, Mk, "bf16")
    assert L16 == L32 and all(np.array_equal(a, b) for a, b in zip(g16, g32))
    params = M.init_params(_u01(3), d_in, width, d_out)
    X = rng.standard_normal((nb, d_in))
    y32, _ = M.forward(params, X)
    y16, _ = M.forward(params, X, "bf16")
    d = np.abs(y16 - y32).max() / np.abs(y32).max()
    assert 1e-5 < d < 5e-2
