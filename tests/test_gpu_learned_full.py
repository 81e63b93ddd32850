"""The learned-interpolation workload at its full size: the network is trained on the GPU on the
exact local solves of 200 seeded 32^3 meshes with alpha = 10^U(-4,4) per element (about 2.2M
samples), then evaluated on a 96^3 mesh with an unseen random jump field against the exact local
solves on convergence factor, setup time and solve time.  Checked: training lowers the loss; the
learned setup either keeps the network with a factor within 10% of the exact one or falls back to
the exact hierarchy; both hierarchies solve to the 1e-8 FP64 relative residual."""
import os
import time

import pytest

import workloads as W
from workloads import fields

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


def test_learned_interpolation_full_size(amgh):
    import torch
    m = amgh.amgh_mlp_create(0)
    t0 = time.perf_counter()
    # the samples need the finest P only: no launch-mode tuning for the 200 training hierarchies
    old = os.environ.get("AMGH_TUNE")
    os.environ["AMGH_TUNE"] = "0"
    try:
        for s in range(200):
            p = W.hex_problem(32, fields.log_uniform(32, 500 + s), 1.0)
            h = amgh.amgh_setup(p["A"], p["G"])
            amgh.amgh_mlp_add_samples(m, h)
            amgh.amgh_destroy(h)
    finally:
        if old is None:
            del os.environ["AMGH_TUNE"]
        else:
            os.environ["AMGH_TUNE"] = old
    t_data = time.perf_counter() - t0
    N = amgh.amgh_mlp_num_samples(m)
    t0 = time.perf_counter()
    losses = [amgh.amgh_mlp_train(m, 1, 512, 1e-3, 10000 + e) for e in range(8)]
    t_train = time.perf_counter() - t0
    print("training set: %d samples from 200 meshes in %.1f s; 8 epochs in %.1f s, loss %.4f -> %.4f"
          % (N, t_data, t_train, losses[0], losses[-1]))
    assert N > 2_000_000
    assert losses[-1] < losses[0]

    p = W.hex_problem(96, fields.random_jump(96, 3, 900), 1.0)
    f = torch.tensor(fields.rhs(p["ndof"], 9), device="cuda")
    amgh.amgh_destroy(amgh.amgh_setup(p["A"], p["G"]))   # fills the launch-mode tuning cache
    out = {}
    variants = [("exact", {}), ("learned", {"interp": amgh.AMGH_INTERP_LEARNED, "mlp": m})]
    for name, kw in variants + [("learned, stored rho", None)]:
        if kw is None:   # deployment: the exact factor is a stored calibration, not re-measured
            kw = {"interp": amgh.AMGH_INTERP_LEARNED, "mlp": m, "rho_ref": out["learned"][0]["rho_exact"]}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = amgh.amgh_setup(p["A"], p["G"], **kw)
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        info = amgh.amgh_info(h)
        x = torch.zeros_like(f)
        t0 = time.perf_counter()
        it, rel, ok = amgh.amgh_pcg_solve(h, f, x, 1e-8, 1000)
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t0
        out[name] = (info, it, rel, ok, t_setup, t_solve)
        print("%s: interpolation kept %s, rho %.4f (exact %.4f), finest P filled in %.1f ms; setup %.2f s, "
              "PCG %d iterations in %.2f s"
              % (name, "learned" if info["interp_used"] == amgh.AMGH_INTERP_LEARNED else "exact", info["rho"],
                 info["rho_exact"], info["interp_ms"], t_setup, it, t_solve))
        assert ok and rel <= 1e-8
        amgh.amgh_destroy(h)
    info = out["learned"][0]
    if info["interp_used"] == amgh.AMGH_INTERP_LEARNED:
        assert info["rho"] <= 1.1 * info["rho_exact"]
    else:
        assert out["learned"][1] == out["exact"][1]     # the fallback is the exact hierarchy
