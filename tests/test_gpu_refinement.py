"""The refinement-based coarse variables ("Ref", Sec. 3) and the geometric Nedelec interpolation
("Geo", the comparison of Sec. 5) on the GPU against the oracle, through the C-ABI: structure
bit-exact on every level, level matrices and P within the same tolerances as the algebraic
hierarchy's (Geo's P is set, not solved: exact), the V-cycle within 4x the largest level
tolerance, PCG within +-1 iteration."""
import numpy as np
import pytest

import workloads as W
from oracle import amg as O
from test_gpu_parity import level_tols, rel, vcycle_tol

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


CASES = [("hex8_block", 8, "local"), ("hex8_block", 8, "geometric"),
         ("hex16_checker", 16, "local"), ("hex16_checker", 16, "geometric")]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "%s-%s" % (c[0], "Geo" if c[2] == "geometric" else "Ref"))
def ref_pair(request, amgh):
    name, n, interp = request.param
    p = W.make_config(name) if name != "hex8_block" else W.hex_problem(8, W.fields.checkerboard(8, 4), 1e-2)
    if "f" not in p:
        p["f"] = W.fields.rhs(p["ndof"], 0)
    H = O.setup(p["A"], p["G"], splitting="refinement", mesh_n=n, interp=interp)
    kw = dict(coarsening=amgh.AMGH_COARSEN_REFINEMENT, mesh_n=n)
    if interp == "geometric":
        kw["interp"] = amgh.AMGH_INTERP_GEOMETRIC
    h = amgh.amgh_setup(p["A"], p["G"], **kw)
    return name, interp, p, H, h


def test_hierarchy_matches_oracle(amgh, ref_pair):
    name, interp, p, H, h = ref_pair
    info = amgh.amgh_info(h)
    assert info["n"] == [L["A"].shape[0] for L in H]
    if interp == "geometric":
        assert info["interp_used"] == amgh.AMGH_INTERP_GEOMETRIC
    tols = level_tols(H)
    for l in range(len(H)):
        A = amgh.amgh_level_matrix(h, l, 0)
        np.testing.assert_array_equal(A.indptr, H[l]["A"].indptr)
        np.testing.assert_array_equal(A.indices, H[l]["A"].indices)
        assert rel(A.data, H[l]["A"].data, "%s %s A_%d" % (name, interp, l)) < tols[l]["A"]
        if l == len(H) - 1:
            break
        s = amgh.amgh_level_structure(h, l)
        cz = H[l]["coarsening"]
        np.testing.assert_array_equal(s["edges"], np.array([[e[0], int(e[1]), e[2], int(e[3]), e[4], e[5], e[6]]
                                                            for e in cz["edges"]], np.int32))
        np.testing.assert_array_equal(s["patch_idx"], np.concatenate(cz["patches"]))
        np.testing.assert_array_equal(s["colour"], H[l]["colour"])
        P = amgh.amgh_level_matrix(h, l, 1)
        np.testing.assert_array_equal(P.indptr, cz["P"].indptr)
        np.testing.assert_array_equal(P.indices, cz["P"].indices)
        if interp == "geometric":
            np.testing.assert_array_equal(P.data, cz["P"].data)
        else:
            assert rel(P.data, cz["P"].data, "%s %s P_%d" % (name, interp, l)) < tols[l]["P"]


def test_vcycle_and_pcg_match_oracle(amgh, ref_pair):
    import torch
    name, interp, p, H, h = ref_pair
    n = p["ndof"]
    r = W.uniform("probe", 100, n)
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    amgh.amgh_vcycle(h, cuda(r), z)
    tv = vcycle_tol(level_tols(H))
    assert rel(z.cpu().numpy(), O.vcycle(H, r), "%s %s vcycle (tol %.1e)" % (name, interp, tv)) < tv
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    it, relres, ok = amgh.amgh_pcg_solve(h, cuda(p["f"]), x, 1e-8, 500)
    _, ito, _ = O.pcg(H, p["f"], tol=1e-8, maxit=500)
    print("%s %s PCG iterations gpu %d oracle %d" % (name, interp, it, ito))
    assert ok and abs(it - ito) <= 1
