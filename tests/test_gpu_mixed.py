"""Mixed precision: the hierarchy and V-cycle stored in FP32 or BF16 (FP32 accumulation) as the
preconditioner of FP64 flexible CG.  The outer residual, SpMV and dots stay FP64, so the method
must still reach a 1e-8 relative residual; the error against the FP64 oracle is stated per result."""
import numpy as np
import pytest

import workloads as W
from oracle import amg as O

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


def cuda(x):
    import torch
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("prec,u", [("f32", 2.0 ** -24), ("bf16", 2.0 ** -9)])
@pytest.mark.parametrize("case", ["hex8_unit", "hex16_checker"])
def test_mixed_vcycle_and_fcg(amgh, prec, u, case):
    import torch
    p = W.make_config(case)
    code = {"f32": amgh.AMGH_F32, "bf16": amgh.AMGH_BF16}[prec]
    h64 = amgh.amgh_setup(p["A"], p["G"])
    h = amgh.amgh_setup(p["A"], p["G"], precision=code)
    H = O.setup(p["A"], p["G"], coarse_size=100)
    info = amgh.amgh_info(h)
    print("mixed %s %s level precisions %s block kappa %s" %
          (case, prec, info["precision"], ["%.1e" % k for k in info["block_kappa"]]))
    # the policy: reduced precision only where kappa * u <= 1/4
    for q, k in zip(info["precision"][:-1], info["block_kappa"][:-1]):
        if q == amgh.AMGH_BF16:
            assert k * 2.0 ** -8 <= 0.25
        elif q == amgh.AMGH_F32:
            assert k * 2.0 ** -24 <= 0.25
        else:
            assert k * 2.0 ** -24 > 0.25 or prec == "f64"
    assert any(q != amgh.AMGH_F64 for q in info["precision"])
    # same structure in every precision
    s64, s = amgh.amgh_level_structure(h64, 0), amgh.amgh_level_structure(h, 0)
    assert np.array_equal(s64["edges"], s["edges"])
    # V-cycle against the FP64 oracle: error of the reduced-precision preconditioner, reported
    r = W.uniform("probe", 7, p["ndof"])
    z = torch.zeros(p["ndof"], dtype=torch.float64, device="cuda")
    amgh.amgh_vcycle(h, cuda(r), z)
    zo = O.vcycle(H, r)
    A = p["A"]
    e = z.cpu().numpy() - zo
    err_A = np.sqrt(e @ (A @ e) / (zo @ (A @ zo)))
    # the per-level bound 8 ((2C-1) kappa u + u) of test_gpu_mixed_parity.py (1-norm condition
    # estimates here), four times its largest value for the V-cycle, in the max norm
    U = {0: 2.0 ** -53, 1: 2.0 ** -24, 2: 2.0 ** -8}
    tv = 4 * max(8 * (2 * c * k * U[q] + U[q]) for q, c, k in
                 zip(info["precision"][:-1], info["ncolours"][:-1], info["block_kappa"][:-1]))
    err_max = float(np.abs(e).max() / np.abs(zo).max())
    print("mixed %s %s V-cycle vs FP64 oracle: A-norm rel err %.3e, max-norm %.3e (bound %.2e)"
          % (case, prec, err_A, err_max, tv))
    assert err_max < tv
    # flexible CG reaches the FP64 tolerance
    f = p["f"]
    x = torch.zeros(p["ndof"], dtype=torch.float64, device="cuda")
    it, rel, ok = amgh.amgh_pcg_solve(h, cuda(f), x, 1e-8, 500)
    xo, ito, _ = O.pcg(H, f, tol=1e-8)
    xs = x.cpu().numpy()
    d = xs - xo
    sol_err = np.sqrt(d @ (A @ d) / (xo @ (A @ xo)))
    print("mixed %s %s FCG iterations %d (FP64 oracle PCG %d), solution A-norm rel err %.3e" %
          (case, prec, it, ito, sol_err))
    assert ok and rel <= 1e-8
    assert it <= 2 * ito + 5
    assert sol_err < 1e-5
