"""Learned interpolation weights on the GPU: the network's initial weights, features, forward pass,
gradients and first Adam step against the FP64 oracle; training on exact local solves; the learned
setup with its convergence-factor fallback; and what the trained network gains over the exact
local solves (fill time of the finest P) and over an untrained network (convergence factor)."""
import numpy as np
import pytest

import workloads as W
from workloads import fields
from oracle import amg as O
from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amgh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2602_23613_gb300 import build, amgh as mod
    build.build()
    mod.load()
    return mod


def oracle_params(seed):
    return M.init_params(lambda count, offset=0: W.uniform01("mlp", seed, count, offset))


def flat(params):
    return np.concatenate([p.ravel() for p in params])


def unflat(v, ref):
    out, o = [], 0
    for p in ref:
        out.append(np.asarray(v[o:o + p.size], dtype=np.float64).reshape(p.shape))
        o += p.size
    return out


def oracle_samples(A, G):
    cz = O.coarsen(A, G)
    X, T, Mk = [], [], []
    for e, pt in zip(cz["edges"], cz["patches"]):
        f, m = M.patch_features(A, e, pt)
        X.append(f)
        Mk.append(m)
        T.append(M.patch_target(A, e, pt))
    return cz, np.array(X), np.array(T), np.array(Mk)


@pytest.fixture(scope="module")
def logu12():
    p = W.hex_problem(12, fields.log_uniform(12, 0), 1.0)
    cz, X, T, Mk = oracle_samples(p["A"], p["G"])
    return p, cz, X, T, Mk


def test_initial_weights_match_oracle(amgh):
    m = amgh.amgh_mlp_create(5)
    got = amgh.amgh_mlp_params(m)
    ref = flat(oracle_params(5)).astype(np.float32)
    np.testing.assert_array_equal(got, ref)


def test_features_and_targets_match_oracle(amgh, logu12):
    p, cz, X, T, Mk = logu12
    h = amgh.amgh_setup(p["A"], p["G"])
    Xg, Tg, Mg = amgh.amgh_mlp_features(h)
    assert Xg.shape == X.shape
    np.testing.assert_array_equal(Mg, Mk.astype(np.float32))
    # features are FP64 values rounded to FP32 on both sides of one log1p
    np.testing.assert_allclose(Xg, X, rtol=2e-6, atol=1e-7)
    np.testing.assert_allclose(Tg, T, rtol=0, atol=1e-6 * np.abs(T).max())


def test_forward_and_gradients_match_oracle(amgh, logu12):
    _, _, X, T, Mk = logu12
    m = amgh.amgh_mlp_create(9)
    params = unflat(amgh.amgh_mlp_params(m), oracle_params(9))
    X32, T32, M32 = X.astype(np.float32), T.astype(np.float32), Mk.astype(np.float32)
    Xd, Td, Md = (a.astype(np.float64) for a in (X32, T32, M32))
    y_ref, _ = M.forward(params, Xd)
    y = amgh.amgh_mlp_predict(m, X32)
    assert np.abs(y - y_ref).max() <= 1e-5 * max(1.0, np.abs(y_ref).max())
    nb = 200
    L, g = amgh.amgh_mlp_loss_grad(m, X32[:nb], T32[:nb], M32[:nb])
    L_ref, g_ref = M.backward(params, Xd[:nb], Td[:nb], Md[:nb])
    g_ref = flat(g_ref)
    print("loss gpu %.8e oracle %.8e; max gradient error %.3e of max %.3e"
          % (L, L_ref, np.abs(g - g_ref).max(), np.abs(g_ref).max()))
    assert abs(L - L_ref) <= 1e-5 * L_ref
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()


def test_first_training_step_matches_oracle_adam(amgh, logu12):
    """One epoch whose single batch holds every sample is one Adam step with the full gradient."""
    p, _, X, T, Mk = logu12
    h = amgh.amgh_setup(p["A"], p["G"])
    m = amgh.amgh_mlp_create(4)
    amgh.amgh_mlp_add_samples(m, h)
    N = amgh.amgh_mlp_num_samples(m)
    assert N == len(X)
    p0 = amgh.amgh_mlp_params(m)
    lr = 1e-3
    amgh.amgh_mlp_train(m, 1, N, lr, 0)
    p1 = amgh.amgh_mlp_params(m)
    params0 = unflat(p0, oracle_params(4))
    _, g = M.backward(params0, X, T, Mk)
    ref = flat(M.adam_step(params0, g, [], lr=lr, t=1))
    g = flat(g)
    sel = np.abs(g) > 1e-3 * np.abs(g).max()
    err = np.abs(p1.astype(np.float64) - ref)[sel].max()
    print("first Adam step: %d of %d parameters with |g| above 1e-3 max, max error %.3e (lr %.0e)"
          % (sel.sum(), len(g), err, lr))
    assert err <= 1e-2 * lr + 1e-7 * np.abs(ref).max()
    assert np.abs(p1 - p0).max() <= lr * (1 + 1e-4)


def test_learned_setup_matches_oracle_pipeline(amgh):
    """With an untrained network kept by force (a huge reference factor), the finest P is the
    network's prediction on Eq. sparseP's pattern and the next level is its Galerkin product."""
    p = W.hex_problem(8, fields.log_uniform(8, 9), 1.0)
    m = amgh.amgh_mlp_create(11)
    params = unflat(amgh.amgh_mlp_params(m), oracle_params(11))
    h = amgh.amgh_setup(p["A"], p["G"], interp=amgh.AMGH_INTERP_LEARNED, mlp=m, rho_ref=1e9)
    info = amgh.amgh_info(h)
    assert info["interp_used"] == amgh.AMGH_INTERP_LEARNED
    H = M.setup_learned(p["A"], p["G"], params)
    P = amgh.amgh_level_matrix(h, 0, 1)
    Pr = H[0]["P"]
    P.sort_indices()
    assert P.nnz == Pr.nnz and np.array_equal(P.indptr, Pr.indptr) and np.array_equal(P.indices, Pr.indices)
    assert np.abs((P - Pr).toarray()).max() <= 1e-5 * max(1.0, abs(Pr).max())
    A1 = amgh.amgh_level_matrix(h, 1, 0)
    assert np.abs((A1 - H[1]["A"]).toarray()).max() <= 1e-4 * abs(H[1]["A"]).max()
    assert [x for x in info["n"]][:2] == [H[0]["A"].shape[0], H[1]["A"].shape[0]]


def test_untrained_network_falls_back_to_exact_solves(amgh):
    p = W.hex_problem(12, fields.log_uniform(12, 1), 1.0)
    m = amgh.amgh_mlp_create(13)
    forced = amgh.amgh_setup(p["A"], p["G"], interp=amgh.AMGH_INTERP_LEARNED, mlp=m, rho_ref=1e9)
    h = amgh.amgh_setup(p["A"], p["G"], interp=amgh.AMGH_INTERP_LEARNED, mlp=m)
    ex = amgh.amgh_setup(p["A"], p["G"])
    fi, info, ei = amgh.amgh_info(forced), amgh.amgh_info(h), amgh.amgh_info(ex)
    print("untrained network: rho %.4f against exact %.4f -> kept %s"
          % (fi["rho"], info["rho_exact"], info["interp_used"] == amgh.AMGH_INTERP_LEARNED))
    assert fi["rho"] > 1.1 * info["rho_exact"]
    assert info["interp_used"] == amgh.AMGH_INTERP_LOCAL
    assert info["n"] == ei["n"] and info["nnz"] == ei["nnz"]
    P, Pe = amgh.amgh_level_matrix(h, 0, 1), amgh.amgh_level_matrix(ex, 0, 1)
    assert np.array_equal(P.data, Pe.data) and np.array_equal(P.indices, Pe.indices)
    # the exact factor measured on the GPU is the oracle's probe factor
    H = O.setup(p["A"], p["G"])
    rho_o = O.probe_factor(H, W.uniform("probe", 0, p["ndof"]))
    assert abs(info["rho_exact"] - rho_o) <= 1e-6 * rho_o


def test_trained_network_gains(amgh):
    """Train on exact local solves of seeded meshes with alpha = 10^U(-4,4) per element; evaluate on
    an unseen random-jump mesh.  The gain over the exact setup is the time to fill the finest P; the
    gain of training is the convergence factor against the untrained network's."""
    import torch
    m = amgh.amgh_mlp_create(0)
    for s in range(6):
        pt = W.hex_problem(12, fields.log_uniform(12, 100 + s), 1.0)
        amgh.amgh_mlp_add_samples(m, amgh.amgh_setup(pt["A"], pt["G"]))
    losses = [amgh.amgh_mlp_train(m, 1, 256, 1e-3, 1000 * e) for e in range(60)]
    print("training on %d samples: epoch loss %.4f -> %.4f" % (amgh.amgh_mlp_num_samples(m), losses[0], losses[-1]))
    assert losses[-1] < 0.8 * losses[0]
    p = W.hex_problem(16, fields.random_jump(16, 3, 7), 1.0)
    ex = amgh.amgh_setup(p["A"], p["G"])
    h = amgh.amgh_setup(p["A"], p["G"], interp=amgh.AMGH_INTERP_LEARNED, mlp=m)
    un = amgh.amgh_setup(p["A"], p["G"], interp=amgh.AMGH_INTERP_LEARNED, mlp=amgh.amgh_mlp_create(1),
                         rho_ref=1e9)
    info, ei, ui = amgh.amgh_info(h), amgh.amgh_info(ex), amgh.amgh_info(un)
    f = torch.tensor(fields.rhs(p["ndof"], 1), device="cuda")
    its = []
    for hh in (ex, h):
        x = torch.zeros_like(f)
        it, rel, ok = amgh.amgh_pcg_solve(hh, f, x, 1e-8, 500)
        assert ok and rel <= 1e-8
        its.append(it)
    print("trained network: kept %s, rho %.4f (exact %.4f, untrained %.4f); PCG iterations %d (exact %d); "
          "finest P filled in %.3f ms (exact local solves %.3f ms)"
          % (info["interp_used"] == amgh.AMGH_INTERP_LEARNED, info["rho"], info["rho_exact"], ui["rho"], its[1],
             its[0], info["interp_ms"], ei["interp_ms"]))
    assert info["interp_used"] == amgh.AMGH_INTERP_LEARNED
    assert info["rho"] <= 1.1 * info["rho_exact"]
    assert info["rho"] < ui["rho"]


def test_bf16_storage_matches_oracle(amgh, logu12):
    """BF16 storage (inputs, weight matrices and hidden activations bfloat16, FP32 accumulation)
    against the oracle's definition on the same FP32 master weights.  The products accumulate in
    FP32 on the GPU and in FP64 in the oracle, so a hidden activation that lies within that
    difference of a bfloat16 rounding boundary may round the other way: one bfloat16 unit (2^-8
    relative) in that activation.  Those rare flips bound the largest difference (1e-2 of max|y|);
    the median difference stays at the FP32 level (1e-4), and the result differs from FP32 storage
    by more than that (the mode is in effect)."""
    _, _, X, T, Mk = logu12
    m = amgh.amgh_mlp_create(9)
    params = unflat(amgh.amgh_mlp_params(m), oracle_params(9))
    X32, T32, M32 = X.astype(np.float32), T.astype(np.float32), Mk.astype(np.float32)
    Xd, Td, Md = (a.astype(np.float64) for a in (X32, T32, M32))
    y32 = amgh.amgh_mlp_predict(m, X32)
    amgh.amgh_mlp_set_precision(m, amgh.AMGH_BF16)
    y = amgh.amgh_mlp_predict(m, X32)
    y_ref, _ = M.forward(params, Xd, "bf16")
    scale = max(1.0, np.abs(y_ref).max())
    err = np.abs(y - y_ref)
    print("BF16 forward: max |y - y_oracle| %.3e, median %.3e, max |y - y_fp32| %.3e (scale %.3e)"
          % (err.max(), np.median(err), np.abs(y - y32).max(), scale))
    assert err.max() <= 1e-2 * scale
    assert np.median(err) <= 1e-4 * scale
    assert np.abs(y - y32).max() >= 1e-4 * scale
    nb = 200
    L, g = amgh.amgh_mlp_loss_grad(m, X32[:nb], T32[:nb], M32[:nb])
    L_ref, g_ref = M.backward(params, Xd[:nb], Td[:nb], Md[:nb], "bf16")
    g_ref = flat(g_ref)
    print("BF16 loss gpu %.8e oracle %.8e; max gradient error %.3e of max %.3e"
          % (L, L_ref, np.abs(g - g_ref).max(), np.abs(g_ref).max()))
    assert abs(L - L_ref) <= 1e-2 * L_ref
    assert np.abs(g - g_ref).max() <= 2e-2 * np.abs(g_ref).max()
    # the masters are untouched; other precisions are refused
    np.testing.assert_array_equal(amgh.amgh_mlp_params(m), flat(params).astype(np.float32))
    with pytest.raises(amgh.AmghError) as e:
        amgh.amgh_mlp_set_precision(m, amgh.AMGH_F64)
    assert e.value.status == amgh.AMGH_ERR_INVALID_ARG


def test_bf16_training_and_learned_setup(amgh, logu12):
    """Training with BF16 storage lowers the loss about as far as FP32 storage does, and a setup
    with the BF16 network runs its fallback test and solves."""
    import torch
    p, _, X, T, Mk = logu12
    h = amgh.amgh_setup(p["A"], p["G"])
    final = {}
    for label, prec in (("fp32", amgh.AMGH_F32), ("bf16", amgh.AMGH_BF16)):
        m = amgh.amgh_mlp_create(4)
        amgh.amgh_mlp_set_precision(m, prec)
        amgh.amgh_mlp_add_samples(m, h)
        losses = [amgh.amgh_mlp_train(m, 1, 256, 1e-3, 100 * e) for e in range(20)]
        final[label] = losses[-1]
        print("%s storage: epoch loss %.5f -> %.5f" % (label, losses[0], losses[-1]))
        assert losses[-1] < 0.9 * losses[0]
    assert final["bf16"] <= 1.25 * final["fp32"]
    hl = amgh.amgh_setup(p["A"], p["G"], interp=amgh.AMGH_INTERP_LEARNED, mlp=m)
    info = amgh.amgh_info(hl)
    f = torch.tensor(fields.rhs(p["ndof"], 1), device="cuda")
    x = torch.zeros_like(f)
    it, rel, ok = amgh.amgh_pcg_solve(hl, f, x, 1e-8, 500)
    print("BF16 network setup: kept %s, rho %.4f (exact %.4f), PCG %d"
          % (info["interp_used"] == amgh.AMGH_INTERP_LEARNED, info["rho"], info["rho_exact"], it))
    assert ok and rel <= 1e-8
