"""Many right-hand sides with one matrix (one matrix read per step for all columns), and the dense
tail of the V-cycle: against the oracle per column and against single-right-hand-side solves."""
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


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.fixture(scope="module")
def checker(amgh):
    p = W.make_config("hex16_checker")
    H = O.setup(p["A"], p["G"], coarse_size=100)
    return p, H


def test_vcycle_multi_matches_oracle_per_column(amgh, checker):
    import torch
    p, H = checker
    h = amgh.amgh_setup(p["A"], p["G"], dense_tail=0)
    k = 5
    R = np.stack([W.uniform("probe", 300 + c, p["ndof"]) for c in range(k)])
    Rd = torch.tensor(R, device="cuda")
    Zd = torch.zeros_like(Rd)
    amgh.amgh_vcycle_multi(h, Rd, Zd)
    Z = Zd.cpu().numpy()
    z1 = torch.zeros(p["ndof"], dtype=torch.float64, device="cuda")
    for c in range(k):
        zo = O.vcycle(H, R[c])
        r = rel(Z[c], zo)
        print("multi vcycle column %d rel err vs oracle %.3e" % (c, r))
        assert r < 2e-5                      # the 16^3 checkerboard's kappa-derived V-cycle bound
        amgh.amgh_vcycle(h, Rd[c].contiguous(), z1)
        assert rel(Z[c], z1.cpu().numpy()) < 2e-5


@pytest.mark.parametrize("k", [8, 33, 65])
def test_pcg_multi_matches_single(amgh, checker, k):
    import torch
    p, H = checker
    h = amgh.amgh_setup(p["A"], p["G"])
    F = np.stack([W.fields.rhs(p["ndof"], 100 + c) for c in range(k)])
    Fd = torch.tensor(F, device="cuda")
    Xd = torch.zeros_like(Fd)
    its, rels, ok = amgh.amgh_pcg_solve_multi(h, Fd, Xd, 1e-8, 300)
    assert ok and max(rels) <= 1e-8
    A = p["A"]
    x1 = torch.zeros(p["ndof"], dtype=torch.float64, device="cuda")
    for c in range(0, k, 7):
        x1.zero_()
        it1, rel1, ok1 = amgh.amgh_pcg_solve(h, Fd[c].contiguous(), x1, 1e-8, 300)
        assert abs(it1 - its[c]) <= 1, (c, it1, its[c])
        d = Xd[c].cpu().numpy() - x1.cpu().numpy()
        xs = x1.cpu().numpy()
        assert np.sqrt(d @ (A @ d)) <= 1e-6 * np.sqrt(xs @ (A @ xs))
    print("multi k=%d iterations %s" % (k, its))
    # host arrays through the same entry point
    Xh = np.zeros_like(F)
    its2, _, ok2 = amgh.amgh_pcg_solve_multi(h, F, Xh, 1e-8, 300)
    assert ok2 and its2 == its


def test_dense_tail_matches_full_recursion(amgh, checker):
    import torch
    p, H = checker
    h0 = amgh.amgh_setup(p["A"], p["G"], dense_tail=0)
    h1 = amgh.amgh_setup(p["A"], p["G"])
    info = amgh.amgh_info(h1)
    assert info["dense_tail"] >= 1 and amgh.amgh_info(h0)["dense_tail"] == -1
    r = torch.tensor(W.uniform("probe", 9, p["ndof"]), device="cuda")
    z0, z1 = torch.zeros_like(r), torch.zeros_like(r)
    amgh.amgh_vcycle(h0, r, z0)
    amgh.amgh_vcycle(h1, r, z1)
    zo = O.vcycle(H, r.cpu().numpy())
    e1, e0 = rel(z1.cpu().numpy(), zo), rel(z0.cpu().numpy(), zo)
    print("dense tail at level %d: V-cycle rel err vs oracle %.3e (full recursion %.3e)" % (info["dense_tail"], e1, e0))
    assert e1 < 2e-5 and e0 < 2e-5
    f = torch.tensor(p["f"], device="cuda")
    x0, x1 = torch.zeros_like(f), torch.zeros_like(f)
    it0, _, _ = amgh.amgh_pcg_solve(h0, f, x0, 1e-8, 300)
    it1, _, _ = amgh.amgh_pcg_solve(h1, f, x1, 1e-8, 300)
    assert abs(it0 - it1) <= 1


def test_vcycle_multi_fp32_levels(amgh, checker):
    """FP32 storage requested: the multi-RHS engine takes each level's storage from the single
    engine (FP64 where the star blocks' kappa u > 1/4, FP32 below), so its V-cycle is the single
    engine's FP32 V-cycle up to FP32 rounding, and both stay close to the FP64 oracle."""
    import torch
    p, H = checker
    h = amgh.amgh_setup(p["A"], p["G"], dense_tail=0, precision=amgh.AMGH_F32)
    info = amgh.amgh_info(h)
    prec = info["precision"][: info["levels"]]
    print("level storage", prec)
    assert amgh.AMGH_F32 in prec
    k = 4
    R = np.stack([W.uniform("probe", 400 + c, p["ndof"]) for c in range(k)])
    Rd = torch.tensor(R, device="cuda")
    Zd = torch.zeros_like(Rd)
    amgh.amgh_vcycle_multi(h, Rd, Zd)
    Z = Zd.cpu().numpy()
    z1 = torch.zeros(p["ndof"], dtype=torch.float64, device="cuda")
    for c in range(k):
        amgh.amgh_vcycle(h, Rd[c].contiguous(), z1)
        e_single = rel(Z[c], z1.cpu().numpy())
        e_oracle = rel(Z[c], O.vcycle(H, R[c]))
        print("FP32 multi vcycle column %d: vs single FP32 %.3e, vs FP64 oracle %.3e" % (c, e_single, e_oracle))
        assert e_single < 1e-4 and e_oracle < 1e-3


@pytest.mark.parametrize("k", [8, 40])
def test_pcg_multi_fp32_matches_single(amgh, checker, k):
    """Flexible block CG with the FP32 multi-RHS V-cycle against flexible single solves with the
    FP32 single-RHS V-cycle: both reach the 1e-8 FP64 residual in nearly the same iterations."""
    import torch
    p, H = checker
    h = amgh.amgh_setup(p["A"], p["G"], precision=amgh.AMGH_F32)
    F = np.stack([W.fields.rhs(p["ndof"], 500 + c) for c in range(k)])
    Fd = torch.tensor(F, device="cuda")
    Xd = torch.zeros_like(Fd)
    its, rels, ok = amgh.amgh_pcg_solve_multi(h, Fd, Xd, 1e-8, 300)
    assert ok and max(rels) <= 1e-8
    A = p["A"]
    x1 = torch.zeros(p["ndof"], dtype=torch.float64, device="cuda")
    for c in range(0, k, 5):
        x1.zero_()
        it1, _, ok1 = amgh.amgh_pcg_solve(h, Fd[c].contiguous(), x1, 1e-8, 300)
        xm = Xd[c].cpu().numpy()
        tr = np.linalg.norm(F[c] - A @ xm) / np.linalg.norm(F[c])
        print("column %d: multi %d iterations, single %d, true residual %.2e" % (c, its[c], it1, tr))
        assert ok1 and abs(it1 - its[c]) <= 2
        # the recurrence reaches 1e-8; the true residual stops at the FP64 floor kappa(A) eps of
        # the 16^3 checkerboard (1.6e-7 with the FP64 V-cycle)
        assert tr < 1e-6
