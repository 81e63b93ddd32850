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
