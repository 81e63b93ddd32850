"""Parity on the benchmark's own workload (64^3 checkerboard, 762,048 DoFs), against the oracle's
values stored by tests/golden/make_oracle_goldens.py (the oracle needs most of an hour for this
size, so its results are stored, not recomputed).  The library is set up exactly as bench.py sets
it up (default parameters), and once more with the commuting correction of the local extension
(interp CONSTRAINED, bench.py --interp constrained) against that form's golden; its P values may
differ by twice the local solves' tolerance plus 1e-13 (see test_gpu_constrained.py).

  * structure: SHA-256 digests of every level's C/F state, coarse edges with signs, coarse nodes,
    patches, star colours and the patterns of A_l and P_l, bit-exact;
  * values: sampled rows of A_l and P_l within max(1e-12, 8 eps kappa) of the oracle, kappa the
    largest condition number of the star or patch blocks the value depends on (stored with the
    golden values);
  * one V-cycle of a seeded vector, on sampled entries, within 4x the largest level tolerance;
  * PCG to 1e-8: iterations within +-1, and the energy f.x within 1e-6 relative (the relative
    A-norm error bound the smaller parity cases use bounds this too:
    |f.x - f.x*| = |(x - x*)^T A x*| <= ||x - x*||_A ||x*||_A).
"""
import hashlib
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDENS = {"local": os.path.join(HERE, "golden", "hex64_checker.json"),
           "constrained": os.path.join(HERE, "golden", "hex64_checker_constrained.json")}
TOL = 1e-12
EPS = np.finfo(np.float64).eps


def digest(arr, dtype):
    return hashlib.sha256(np.ascontiguousarray(np.asarray(arr), dtype=np.dtype(dtype).newbyteorder("<"))
                          .tobytes()).hexdigest()


@pytest.fixture(scope="module", params=list(GOLDENS))
def form(request):
    return request.param


@pytest.fixture(scope="module")
def gold(form):
    return json.load(open(GOLDENS[form]))


@pytest.fixture(scope="module")
def amgh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2602_23613_gb300 import build, amgh as mod
    build.build()
    mod.load()
    return mod


@pytest.fixture(scope="module")
def problem():
    return W.make_config("hex64_checker")


@pytest.fixture(scope="module")
def bench_handle(amgh, problem, form):
    kw = {} if form == "local" else dict(interp=amgh.AMGH_INTERP_CONSTRAINED)
    h = amgh.amgh_setup(problem["A"], problem["G"], **kw)
    return problem, h


def level_tols(gold):
    constrained = gold["params"].get("interp", "local") == "constrained"
    out, prev_p = [], TOL
    for l, g in enumerate(gold["levels"]):
        tp = max(TOL, 8 * EPS * g.get("kappa_patch", 1.0))
        if constrained:
            tp = 2 * tp + 1e-13
        t = dict(smooth=max(TOL, 8 * EPS * g["kappa_star"]), P=tp, A=max(TOL, 2 * prev_p))
        out.append(t)
        prev_p = t["P"] if l == 0 else max(t["P"], t["A"])
    return out


def test_structure_digests_every_level(amgh, bench_handle, gold):
    p, h = bench_handle
    info = amgh.amgh_info(h)
    assert info["n"] == [g["n"] for g in gold["levels"]]
    assert info["nnz"] == [g["nnz"] for g in gold["levels"]]
    # the coarsest level has no smoother in the library (its dense inverse replaces it)
    assert info["ncolours"][:-1] == [g["ncolours"] for g in gold["levels"]][:-1]
    for l, g in enumerate(gold["levels"]):
        d = g["digests"]
        A = amgh.amgh_level_matrix(h, l, 0)
        assert digest(A.indptr, "i4") == d["A_indptr"], l
        assert digest(A.indices, "i4") == d["A_indices"], l
        if l == len(gold["levels"]) - 1:
            break
        s = amgh.amgh_level_structure(h, l)
        assert digest(s["colour"], "i4") == d["colour"], l
        if "cf_state" not in d:
            continue
        assert digest(s["cf_state"], "i1") == d["cf_state"], l
        assert digest(s["edges"].astype(np.int64), "i4") == d["edges"], l
        assert digest(s["coarse_nodes"], "i4") == d["coarse_nodes"], l
        assert digest(s["patch_ptr"], "i4") == d["patch_ptr"], l
        assert digest(s["patch_idx"], "i4") == d["patch_idx"], l
        P = amgh.amgh_level_matrix(h, l, 1)
        assert digest(P.indptr, "i4") == d["P_indptr"], l
        assert digest(P.indices, "i4") == d["P_indices"], l


def _rows_rel(M, sample):
    worst, scale = 0.0, 0.0
    for r, vals in zip(sample["rows"], sample["values"]):
        got = M.data[M.indptr[r]:M.indptr[r + 1]]
        want = np.asarray(vals)
        assert len(got) == len(want)
        worst = max(worst, float(np.abs(got - want).max()) if len(want) else 0.0)
        scale = max(scale, float(np.abs(want).max()) if len(want) else 0.0)
    return worst / scale if scale > 0 else worst


def test_level_values_on_sampled_rows(amgh, bench_handle, gold):
    p, h = bench_handle
    tols = level_tols(gold)
    for l, g in enumerate(gold["levels"]):
        e = _rows_rel(amgh.amgh_level_matrix(h, l, 0), g["A_rows"])
        print("hex64 A_%d sampled rows rel %.3e (tol %.1e)" % (l, e, tols[l]["A"]))
        assert e < tols[l]["A"], (l, e)
        if "P_rows" in g:
            e = _rows_rel(amgh.amgh_level_matrix(h, l, 1), g["P_rows"])
            print("hex64 P_%d sampled rows rel %.3e (tol %.1e)" % (l, e, tols[l]["P"]))
            assert e < tols[l]["P"], (l, e)


def test_vcycle_on_sampled_entries(amgh, bench_handle, gold):
    import torch
    p, h = bench_handle
    n = p["ndof"]
    v = gold["vcycle"]
    r = torch.tensor(W.uniform(v["probe_stream"], v["probe_seed"], n), device="cuda")
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    amgh.amgh_vcycle(h, r, z)
    zs = z.cpu().numpy()
    tv = 4 * max(max(t.values()) for t in level_tols(gold))
    e = float(np.abs(zs[v["idx"]] - np.asarray(v["values"])).max() / v["inf_norm"])
    print("hex64 V-cycle sampled rel %.3e (tol %.1e); inf-norm %.6e vs %.6e" % (e, tv, np.abs(zs).max(), v["inf_norm"]))
    assert e < tv
    assert abs(np.abs(zs).max() - v["inf_norm"]) <= tv * v["inf_norm"]
    assert abs(np.linalg.norm(zs) - v["two_norm"]) <= tv * v["two_norm"]


def test_pcg_iterations_and_energy(amgh, bench_handle, gold):
    import torch
    p, h = bench_handle
    g = gold["pcg"]
    f = torch.tensor(p["f"], device="cuda")
    x = torch.zeros_like(f)
    it, rel, ok = amgh.amgh_pcg_solve(h, f, x, 1e-8, 2000)
    xs = x.cpu().numpy()
    energy = float(p["f"] @ xs)
    print("hex64 PCG iterations gpu %d oracle %d; energy rel diff %.3e"
          % (it, g["iterations"], abs(energy - g["energy"]) / abs(g["energy"])))
    assert ok and rel <= 1e-8
    assert abs(it - g["iterations"]) <= 1
    assert abs(energy - g["energy"]) <= 1e-6 * abs(g["energy"])
