"""Fused residual + restriction (Eq. tl's coarse right-hand side r_c = P^T (f - A y)) computed as
P^T f - W y with W = P^T A, one pass and no fine residual: against the oracle's P.T @ (f - A @ y)
on every level, inside the V-cycle and inside PCG.

Tolerance (componentwise, from the summation error of a dot product): the fused pass sums the
terms of P^T f and of W y in a different order than the oracle's two passes and W's own entries
carry one rounding of their k-term sums, so each coarse entry may differ by at most
  c * eps * (|P^T| |f| + |P^T| |A| |y|)_i,   c = 2 (k_P + k_W + k_A + 2),
k_* the longest row of P^T, W and A."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import amg as O
from test_gpu_parity import level_tols, vcycle_tol

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def amgh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2602_23613_gb300 import build, amgh as mod
    build.build()
    mod.load()
    return mod


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
def fused(request, amgh):
    p = CASES[request.param]()
    cs = 32 if request.param.startswith("tri") else 100
    H = O.setup(p["A"], p["G"], coarse_size=cs)
    h = amgh.amgh_setup(p["A"], p["G"], coarse_size=cs, fuse_restrict=1, dense_tail=0)
    return request.param, p, H, h


def maxrow(M):
    M = sp.csr_matrix(M)
    return int(np.diff(M.indptr).max()) if M.shape[0] else 0


def test_fused_pass_matches_oracle_per_level(amgh, fused):
    import torch
    name, p, H, h = fused
    info = amgh.amgh_info(h)
    assert all(info["fused_rr"][l] == 1 for l in range(len(H) - 1)), info["fused_rr"]
    for l in range(len(H) - 1):
        L = H[l]
        A, P = L["A"], L["P"]
        n, nc = A.shape[0], P.shape[1]
        f = W.uniform("probe", 500 + l, n)
        y = W.uniform("probe", 600 + l, n)
        out = torch.zeros(nc, dtype=torch.float64, device="cuda")
        amgh.amgh_level_apply(h, l, 7, cuda(f), cuda(y), out)
        got = out.cpu().numpy()
        want = P.T @ (f - A @ y)
        PTa = abs(sp.csr_matrix(P.T))
        scale = PTa @ np.abs(f) + PTa @ (abs(A) @ np.abs(y))
        Wm = sp.csr_matrix(P.T @ A)
        c = 2 * (maxrow(P.T) + maxrow(Wm) + maxrow(A) + 2)
        err = np.abs(got - want)
        ratio = float((err / (c * EPS * scale + 1e-300)).max())
        print("fused %s level %d: max |err| / bound %.3f, rel err %.2e" % (name, l, ratio,
                                                                          err.max() / np.abs(want).max()))
        assert ratio <= 1.0, (name, l, ratio)
        # the two-pass path of the same handle: residual (op 1) then restriction (op 4)
        r = torch.zeros(n, dtype=torch.float64, device="cuda")
        amgh.amgh_level_apply(h, l, 1, cuda(f), cuda(y), r)
        two = torch.zeros(nc, dtype=torch.float64, device="cuda")
        amgh.amgh_level_apply(h, l, 4, None, r, two)
        assert float((np.abs(two.cpu().numpy() - got) / (c * EPS * scale + 1e-300)).max()) <= 2.0


def test_vcycle_and_pcg_with_fused_pass(amgh, fused):
    """The whole V-cycle with the fused pass on every level: within the FP64 parity tolerance of
    the oracle's V-cycle (the kappa-scaled bound of the unfused path), and PCG within +-1."""
    import torch
    name, p, H, h = fused
    h2 = amgh.amgh_setup(p["A"], p["G"], coarse_size=32 if name.startswith("tri") else 100, fuse_restrict=0,
                         dense_tail=0)
    assert all(v == 0 for v in amgh.amgh_info(h2)["fused_rr"])
    n = p["ndof"]
    r = W.uniform("probe", 100, n)
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    z2 = torch.zeros_like(z)
    amgh.amgh_vcycle(h, cuda(r), z)
    amgh.amgh_vcycle(h2, cuda(r), z2)
    zo = O.vcycle(H, r)
    e1 = float(np.abs(z.cpu().numpy() - zo).max() / np.abs(zo).max())
    e2 = float(np.abs(z2.cpu().numpy() - zo).max() / np.abs(zo).max())
    tv = vcycle_tol(level_tols(H))
    print("fused %s V-cycle rel err: fused %.2e, apart %.2e (tol %.1e)" % (name, e1, e2, tv))
    assert e1 < tv and e2 < tv
    f = p["f"] if "f" in p else W.fields.rhs(n, 0)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    it, rel, ok = amgh.amgh_pcg_solve(h, cuda(f), x, 1e-8, 300)
    _, ito, _ = O.pcg(H, f, tol=1e-8, maxit=300)
    assert ok and abs(it - ito) <= 1, (it, ito)
    # a handle without W refuses the fused operation
    with pytest.raises(amgh.AmghError) as e:
        amgh.amgh_level_apply(h2, 0, 7, cuda(f), cuda(r), torch.zeros(H[1]["A"].shape[0], dtype=torch.float64,
                                                                     device="cuda"))
    assert e.value.status == amgh.AMGH_ERR_INVALID_ARG
