"""Device-resident PCG (one CUDA graph with a conditional WHILE node) and many independent systems
of uneven size solved by one graph launch: same iterations and the same bits as one-by-one solves,
iterations within +-1 of the oracle's."""
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


def test_device_loop_equals_host_loop(amgh):
    import torch
    p = W.make_config("hex16_checker")
    h = amgh.amgh_setup(p["A"], p["G"])
    f = cuda(p["f"])
    x1 = torch.zeros_like(f)
    it1, rel1, ok1 = amgh.amgh_pcg_solve(h, f, x1, 1e-8, 300)        # device-resident loop
    amgh.amgh_profile(h, 1, "schwarz", 0)                               # forces the host loop
    x2 = torch.zeros_like(f)
    it2, rel2, ok2 = amgh.amgh_pcg_solve(h, f, x2, 1e-8, 300)
    amgh.amgh_profile(h, 0)
    assert ok1 and ok2 and it1 == it2 and rel1 == rel2
    assert torch.equal(x1, x2)
    # a second device solve reuses the captured graph and repeats the bits
    x3 = torch.zeros_like(f)
    it3, rel3, _ = amgh.amgh_pcg_solve(h, f, x3, 1e-8, 300)
    assert it3 == it1 and torch.equal(x3, x1)


def _batch_problems(count):
    probs = []
    for s in range(count):
        n = 6 + int(W.uniform01("sys_n", 1000 + s, 1)[0] * 11)        # 6..16 hexes per side
        k = 1 + int(W.uniform01("sys_k", 1000 + s, 1)[0] * 6)          # jump 10^k, k in 1..6
        alpha = W.fields.random_jump(n, k, 2000 + s, nb=2 if n % 2 == 0 else 1)
        p = W.hex_problem(n, alpha, 1e-2)
        p["f"] = W.fields.rhs(p["ndof"], s)
        probs.append(p)
    return probs


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_of_uneven_systems_in_one_launch(amgh, prec):
    import torch
    code = {"f64": amgh.AMGH_F64, "f32": amgh.AMGH_F32}[prec]
    probs = _batch_problems(8)
    hs = [amgh.amgh_setup(p["A"], p["G"], precision=code) for p in probs]
    fs = [cuda(p["f"]) for p in probs]
    xs = [torch.zeros_like(f) for f in fs]
    its, rels, ok = amgh.amgh_batch_pcg_solve(hs, fs, xs, 1e-8, 300)
    assert ok and all(r <= 1e-8 for r in rels)
    for i, (p, h) in enumerate(zip(probs, hs)):
        x1 = torch.zeros_like(fs[i])
        it1, rel1, _ = amgh.amgh_pcg_solve(h, fs[i], x1, 1e-8, 300)
        assert it1 == its[i] and torch.equal(x1, xs[i]), i
        if prec == "f64":
            H = O.setup(p["A"], p["G"], coarse_size=100)
            _, ito, _ = O.pcg(H, p["f"], tol=1e-8)
            assert abs(ito - its[i]) <= 1, (i, its[i], ito)
    print("batch %s sizes %s iterations %s" % (prec, [p["ndof"] for p in probs], its))


def test_batch_setup_equals_one_by_one(amgh):
    """amgh_batch_setup builds the same hierarchies as amgh_setup one by one: same levels, same
    structure, and (launch choices cached by the one-by-one setups first) bitwise the same PCG
    solves; the wall times of both are printed."""
    import time
    import torch
    probs = _batch_problems(8)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hs1 = [amgh.amgh_setup(p["A"], p["G"]) for p in probs]
    t1 = time.perf_counter()
    hs2 = amgh.amgh_batch_setup([p["A"] for p in probs], [p["G"] for p in probs])
    t2 = time.perf_counter()
    print("batch setup of %d systems: one by one %.1f ms, batch %.1f ms" % (len(probs), 1e3 * (t1 - t0),
                                                                           1e3 * (t2 - t1)))
    for i, (p, a, b) in enumerate(zip(probs, hs1, hs2)):
        ia, ib = amgh.amgh_info(a), amgh.amgh_info(b)
        assert ia["n"] == ib["n"] and ia["nnz"] == ib["nnz"] and ia["fused"] == ib["fused"], i
        sa, sb = amgh.amgh_level_structure(a, 0), amgh.amgh_level_structure(b, 0)
        assert np.array_equal(sa["edges"], sb["edges"]) and np.array_equal(sa["colour"], sb["colour"])
        f = cuda(p["f"])
        xa, xb = torch.zeros_like(f), torch.zeros_like(f)
        ita, _, oka = amgh.amgh_pcg_solve(a, f, xa, 1e-8, 300)
        itb, _, okb = amgh.amgh_pcg_solve(b, f, xb, 1e-8, 300)
        assert oka and okb and ita == itb and torch.equal(xa, xb), i


def test_batch_setup_reports_the_failing_system(amgh):
    import scipy.sparse as sp
    probs = _batch_problems(3)
    bad = sp.csr_matrix(probs[1]["G"], copy=True)
    bad.data[0] = 3.0
    with pytest.raises(amgh.AmghError) as e:
        amgh.amgh_batch_setup([p["A"] for p in probs], [probs[0]["G"], bad, probs[2]["G"]])
    assert e.value.status == amgh.AMGH_ERR_INVALID_ARG
    assert "system 1" in str(e.value)
