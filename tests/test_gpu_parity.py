"""GPU parity of libamgh against the CPU oracle, through the C-ABI.

Structure (C/F splitting, coarse edges, patches, colours, patterns) must be bit-exact on every
level; PCG iteration counts within +-1 of the oracle's at tol 1e-8.  FP64 values must agree to
1e-12 relative (max-norm) per level matrix and per kernel application wherever the arithmetic
allows it: a dense solve with a block of condition number kappa has a forward error of order
kappa * eps in any backward-stable implementation, so two correct implementations may differ by
that much (the oracle itself moves by up to kappa * eps / 2 when its block inverses are swapped
for Cholesky solves).  Node-star blocks contain their node's gradient, an O(beta) mode, so on the
finest level kappa reaches 1e9 for beta = 1e-2; each comparison therefore uses
max(1e-12, 8 eps kappa) with kappa the largest condition number of the dense blocks (star blocks
for the smoother, patch blocks A_pp for P and the Galerkin product) that the compared result
depends on."""
import numpy as np
import pytest

import workloads as W
from oracle import amg as O

pytestmark = pytest.mark.gpu

TOL = 1e-12
EPS = np.finfo(np.float64).eps


def level_tols(H):
    """Per level: tolerance of the smoother (star blocks), of P (patch blocks) and of A_l."""
    out = []
    prev_p = TOL
    for l, L in enumerate(H):
        A = L["A"]
        ks = max((np.linalg.cond(A[b][:, b].toarray()) for b in L["stars"] if len(b)), default=1.0)
        kp = 1.0
        if "coarsening" in L and L["coarsening"].get("patches") is not None:
            kp = max((np.linalg.cond(A[q][:, q].toarray()) for q in L["coarsening"]["patches"] if len(q)),
                     default=1.0)
        out.append(dict(smooth=max(TOL, 8 * EPS * ks), P=max(TOL, 8 * EPS * kp), A=max(TOL, 2 * prev_p)))
        prev_p = out[-1]["P"] if l == 0 else max(out[-1]["P"], out[-1]["A"])
    return out


def vcycle_tol(tols):
    return 4 * max(max(t.values()) for t in tols)


@pytest.fixture(scope="module")
def amgh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2602_23613_gb300 import build, amgh as mod
    build.build()
    mod.load()
    return mod


def rel(a, b, what=""):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.abs(b).max()
    r = float(np.abs(a - b).max() / (s if s > 0 else 1.0))
    if what:
        print("parity %-40s rel %.3e" % (what, r))
    return r


def cuda(x):
    import torch
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


CASES = {
    "hex8_unit": lambda: W.make_config("hex8_unit"),
    "hex12_lognormal": lambda: W.hex_problem(12, W.fields.log_uniform(12, 3, lo=-2, hi=2), 0.1),
    "hex16_checker": lambda: W.make_config("hex16_checker"),
    "tri32": lambda: W.tri_problem(32, 1.0, 0.01),
}


@pytest.fixture(scope="module", params=list(CASES))
def pair(request, amgh):
    p = CASES[request.param]()
    cs = 32 if request.param.startswith("tri") else 100
    H = O.setup(p["A"], p["G"], coarse_size=cs)
    h = amgh.amgh_setup(p["A"], p["G"], coarse_size=cs)
    return request.param, p, H, h, level_tols(H)


def test_hierarchy_structure_and_values(amgh, pair):
    name, p, H, h, tols = pair
    info = amgh.amgh_info(h)
    assert info["n"] == [L["A"].shape[0] for L in H]
    for l in range(len(H)):
        A = amgh.amgh_level_matrix(h, l, 0)
        Ao = H[l]["A"]
        np.testing.assert_array_equal(A.indptr, Ao.indptr)
        np.testing.assert_array_equal(A.indices, Ao.indices)
        assert rel(A.data, Ao.data, "%s A_%d" % (name, l)) < tols[l]["A"], (name, l)
        if l == len(H) - 1:
            break
        s = amgh.amgh_level_structure(h, l)
        cz = H[l]["coarsening"]
        state = np.full(cz["Gt"].shape[1], 2, np.int8)
        state[cz["cG"]] = 1
        state[cz["B"]] = 1
        np.testing.assert_array_equal(s["cf_state"], state)
        np.testing.assert_array_equal(s["edges"], np.array([list(e) for e in cz["edges"]], np.int32))
        np.testing.assert_array_equal(s["patch_idx"], np.concatenate(cz["patches"]))
        np.testing.assert_array_equal(s["colour"], H[l]["colour"])
        P = amgh.amgh_level_matrix(h, l, 1)
        np.testing.assert_array_equal(P.indptr, cz["P"].indptr)
        np.testing.assert_array_equal(P.indices, cz["P"].indices)
        assert rel(P.data, cz["P"].data, "%s P_%d" % (name, l)) < tols[l]["P"], (name, l)


def test_level_kernels(amgh, pair):
    """Each V-cycle step on each level against the oracle's step on the same level."""
    import torch
    name, p, H, h, tols = pair
    for l in range(len(H)):
        L = H[l]
        n = L["A"].shape[0]
        x = W.uniform("probe", 10 + l, n)
        f = W.uniform("probe", 40 + l, n)
        y = torch.zeros(n, dtype=torch.float64, device="cuda")
        if l == len(H) - 1:
            amgh.amgh_level_apply(h, l, 6, None, cuda(f), y)
            from scipy.linalg import cho_solve
            assert rel(y.cpu().numpy(), cho_solve(L["chol"], f)) < max(tols[l]["A"], 8 * EPS * np.linalg.cond(L["A"].toarray()))
            break
        amgh.amgh_level_apply(h, l, 0, None, cuda(x), y)
        assert rel(y.cpu().numpy(), L["A"] @ x) < tols[l]["A"], (name, l, "spmv")
        amgh.amgh_level_apply(h, l, 1, cuda(f), cuda(x), y)
        assert rel(y.cpu().numpy(), f - L["A"] @ x) < tols[l]["A"], (name, l, "residual")
        amgh.amgh_level_apply(h, l, 2, cuda(f), cuda(x), y)
        assert rel(y.cpu().numpy(), O.smooth_pre(L, f, x.copy()), "%s pre_%d (tol %.1e)" % (name, l, tols[l]["smooth"])) < tols[l]["smooth"], (name, l, "pre-step")
        amgh.amgh_level_apply(h, l, 3, cuda(f), cuda(x), y)
        assert rel(y.cpu().numpy(), O.smooth_post(L, f, x.copy()), "%s post_%d" % (name, l)) < tols[l]["smooth"], (name, l, "post-step")
        nc = H[l + 1]["A"].shape[0]
        yc = torch.zeros(nc, dtype=torch.float64, device="cuda")
        amgh.amgh_level_apply(h, l, 4, None, cuda(x), yc)
        assert rel(yc.cpu().numpy(), L["P"].T @ x) < tols[l]["P"], (name, l, "restrict")
        e = W.uniform("probe", 70 + l, nc)
        y0 = cuda(f)
        amgh.amgh_level_apply(h, l, 5, None, cuda(e), y0)
        assert rel(y0.cpu().numpy(), f + L["P"] @ e) < tols[l]["P"], (name, l, "prolong")


def test_vcycle_matches_oracle(amgh, pair):
    import torch
    name, p, H, h, tols = pair
    n = p["ndof"]
    tv = vcycle_tol(tols)
    for seed in (0, 1):
        r = W.uniform("probe", 100 + seed, n)
        z = torch.zeros(n, dtype=torch.float64, device="cuda")
        amgh.amgh_vcycle(h, cuda(r), z)
        zo = O.vcycle(H, r)
        assert rel(z.cpu().numpy(), zo, "%s vcycle (tol %.1e)" % (name, tv)) < tv, name
    # host buffers through the same entry point give the same bits
    zh = np.zeros(n)
    amgh.amgh_vcycle(h, r, zh)
    np.testing.assert_array_equal(zh, z.cpu().numpy())


def test_pcg_matches_oracle(amgh, pair):
    import torch
    name, p, H, h, tols = pair
    f = p["f"] if "f" in p else W.fields.rhs(p["ndof"], 0)
    x = torch.zeros(p["ndof"], dtype=torch.float64, device="cuda")
    it, relres, ok = amgh.amgh_pcg_solve(h, cuda(f), x, 1e-8, 300)
    xo, ito, hist = O.pcg(H, f, tol=1e-8, maxit=300)
    print("parity %s PCG iterations gpu %d oracle %d" % (name, it, ito))
    assert ok and abs(it - ito) <= 1, (name, it, ito)
    assert relres <= 1e-8
    xs = x.cpu().numpy()
    A = p["A"]
    e = xs - xo
    assert np.sqrt(e @ (A @ e)) <= 1e-6 * np.sqrt(xo @ (A @ xo))
    # host buffers: same answer, same count
    xh = np.zeros(p["ndof"])
    it2, rel2, ok2 = amgh.amgh_pcg_solve(h, f, xh, 1e-8, 300)
    assert it2 == it and np.array_equal(xh, xs)


def test_amg_iteration_matches_oracle(amgh):
    p = W.tri_problem(16, 1.0, 0.01)
    n = p["ndof"]
    b = np.arange(1, n + 1, dtype=float)
    x0 = W.uniform("x0", 0, n)
    H = O.setup(p["A"], p["G"], coarse_size=32)
    h = amgh.amgh_setup(p["A"], p["G"], coarse_size=32)
    x = x0.copy()
    it, relres, ok = amgh.amgh_amg_solve(h, b, x, 1e-8, 200)
    _, ito, _ = O.amg_iterate(H, b, x0=x0)
    assert ok and abs(it - ito) <= 1
    x = x0.copy()
    it, relres, ok = amgh.amgh_pcg_solve(h, b, x, 1e-8, 200)
    _, ito, _ = O.pcg(H, b, x0=x0)
    assert ok and abs(it - ito) <= 1


def test_errors_are_statuses(amgh):
    p = W.hex_problem(4, 1.0, 1.0)
    G = p["G"].tolil()
    G[0, 0] = 3.0
    with pytest.raises(amgh.AmghError) as e:
        amgh.amgh_setup(p["A"], G.tocsr())
    assert e.value.status == amgh.AMGH_ERR_INVALID_ARG
    # a non-SPD operator is reported by the factorisations, not by a fault
    A = -W.hex_problem(6, 1.0, 1.0)["A"]
    with pytest.raises(amgh.AmghError) as e:
        amgh.amgh_setup(A, W.hex_problem(6, 1.0, 1.0)["G"])
    assert e.value.status == amgh.AMGH_ERR_NOT_SPD
    # maxit reached: NOT_CONVERGED with the iterate returned
    q = W.make_config("hex8_unit")
    h = amgh.amgh_setup(q["A"], q["G"])
    x = np.zeros(q["ndof"])
    it, relres, ok = amgh.amgh_pcg_solve(h, q["f"], x, 1e-14, 2)
    assert not ok and it == 2 and relres < 1


@pytest.fixture(scope="module")
def full(amgh):
    p = W.make_config("hex64_checker")
    h = amgh.amgh_setup(p["A"], p["G"])
    return p, h


def test_full_size_sampled(amgh, full):
    """The bench workload (64^3 checkerboard): the residual kernel on sampled rows against the
    oracle's formula, structural invariants of the hierarchy, and convergence with the true
    residual checked on the host."""
    import torch
    p, h = full
    A = p["A"]
    n = p["ndof"]
    info = amgh.amgh_info(h)
    assert info["n"][0] == n and info["levels"] >= 4
    rng = np.random.default_rng(0)
    x = W.uniform("probe", 5, n)
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    amgh.amgh_level_apply(h, 0, 1, cuda(p["f"]), cuda(x), y)
    rows = rng.choice(n, 2000, replace=False)
    ref = p["f"][rows] - A[rows] @ x
    assert rel(y.cpu().numpy()[rows], ref) < TOL
    s = amgh.amgh_level_structure(h, 0)
    edges = s["edges"]
    assert len(np.unique(edges[:, 5])) == len(edges)                 # one path per middle node
    ext = np.concatenate([edges[:, 0], edges[:, 2]])
    assert len(np.unique(ext)) == len(ext)                            # distinct pairing
    # the structure, the level matrices, a V-cycle and the PCG count against the oracle's own
    # hierarchy of this workload: tests/test_gpu_bench_golden.py
    # convergence through the public entry point, with the true residual checked on the host
    xs = np.zeros(n)
    it, relres, ok = amgh.amgh_pcg_solve(h, p["f"], xs, 1e-8, 500)
    assert ok and relres <= 1e-8
    true_rel = np.linalg.norm(p["f"] - A @ xs) / np.linalg.norm(p["f"])
    assert true_rel < 1e-5
