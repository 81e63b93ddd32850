"""CPU tests of the C-ABI library: it loads, exports every declared symbol, validates inputs, and
its host graph steps (Alg. 1-3, patches, smoother stars/colours, symbolic Galerkin pattern)
reproduce the oracle's structure bit for bit.  No GPU call is made."""
import ctypes
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import amg as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def amgh():
    from paper_2602_23613_gb300 import build, amgh as mod
    build.build()
    mod.load()
    return mod


def test_exports_every_declared_symbol(amgh):
    header = open(os.path.join(ROOT, "include", "amgh.h")).read()
    declared = set(re.findall(r"^\s*(?:amgh_status|void|int64_t|const char\*)\s+(amgh_\w+)\s*\(", header, re.M))
    assert len(declared) >= 14
    lib = ctypes.CDLL(amgh.lib_path())
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(amgh.EXPORTS)


def _oracle_structure(p):
    cz = O.coarsen(p["A"], p["G"])
    state = np.full(cz["Gt"].shape[1], 2, np.int8)
    state[cz["cG"]] = 1
    state[cz["B"]] = 1
    edges = np.array([list(e) for e in cz["edges"]], np.int64)
    pptr = np.concatenate([[0], np.cumsum([len(x) for x in cz["patches"]])])
    return cz, state, edges, pptr


@pytest.mark.parametrize("maker", [lambda: W.hex_problem(8, 1.0, 1.0),
                                   lambda: W.hex_problem(10, W.fields.log_uniform(10, 3), 0.1),
                                   lambda: W.make_config("hex16_checker"),
                                   lambda: W.tri_problem(16, 1.0, 0.01),
                                   lambda: W.quad_problem(10, 1.0, 0.01)])
def test_host_structure_matches_oracle(amgh, maker):
    p = maker()
    h = amgh.amgh_setup_host_structure(p["A"], p["G"])
    s = amgh.amgh_level_structure(h, 0)
    cz, state, edges, pptr = _oracle_structure(p)
    np.testing.assert_array_equal(s["cf_state"], state)
    np.testing.assert_array_equal(s["edges"].astype(np.int64), edges)
    np.testing.assert_array_equal(s["coarse_nodes"], cz["coarse_nodes"])
    np.testing.assert_array_equal(s["patch_ptr"], pptr)
    np.testing.assert_array_equal(s["patch_idx"], np.concatenate(cz["patches"]))
    np.testing.assert_array_equal(s["colour"], O.colour_stars(p["A"], p["G"]))
    P = amgh.amgh_level_matrix(h, 0, 1)
    np.testing.assert_array_equal(P.indptr, cz["P"].indptr)
    np.testing.assert_array_equal(P.indices, cz["P"].indices)
    # the exterior rows of P are R^T exactly (Eq. sparseP)
    ext = np.zeros(p["ndof"], bool)
    ext[edges[:, 0]] = ext[edges[:, 2]] = True
    np.testing.assert_array_equal(P[ext].toarray(), cz["P"][ext].toarray())
    Ac = amgh.amgh_level_matrix(h, 0, 3)
    Aco = O.galerkin(p["A"], cz["P"])
    np.testing.assert_array_equal(Ac.indptr, Aco.indptr)
    np.testing.assert_array_equal(Ac.indices, Aco.indices)
    Gc = cz["Gc"]
    np.testing.assert_array_equal(np.diff(Gc.indptr) >= 1, True)


@pytest.mark.slow
def test_host_structure_matches_oracle_32(amgh):
    test_host_structure_matches_oracle(amgh, lambda: W.make_config("hex32_checker"))


def test_input_validation(amgh):
    p = W.hex_problem(4, 1.0, 1.0)
    G = p["G"].tolil()
    G[0, 0] = 2.0
    with pytest.raises(amgh.AmghError) as e:
        amgh.amgh_setup_host_structure(p["A"], G.tocsr())
    assert e.value.status == amgh.AMGH_ERR_INVALID_ARG
    G = p["G"].tolil()
    r = G.rows[5]
    G[5, r[0]] = G[5, r[1]] if len(r) > 1 else G[5, r[0]]
    if len(r) > 1:
        with pytest.raises(amgh.AmghError):
            amgh.amgh_setup_host_structure(p["A"], G.tocsr())
    A = p["A"][:, :-1]
    with pytest.raises(amgh.AmghError):
        amgh.amgh_setup_host_structure(A, p["G"])
    # unsorted columns are rejected
    A = p["A"].copy()
    A.has_sorted_indices = True
    i0 = A.indptr[3]
    A.indices[i0], A.indices[i0 + 1] = A.indices[i0 + 1], A.indices[i0]
    from paper_2602_23613_gb300.amgh import _csr, amgh_csr
    keep = []
    ca = amgh_csr()
    rp = np.ascontiguousarray(A.indptr, np.int32)
    ci = np.ascontiguousarray(A.indices, np.int32)
    va = np.ascontiguousarray(A.data, np.float64)
    ca.nrows = ca.ncols = A.shape[0]
    ca.nnz = A.nnz
    ca.row_ptr, ca.col, ca.val, ca.on_device = rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0
    cg = _csr(p["G"], keep)
    out = ctypes.c_void_p()
    st = amgh.load().amgh_setup_host_structure(ctypes.byref(ca), ctypes.byref(cg), None, ctypes.byref(out))
    assert st == amgh.AMGH_ERR_INVALID_ARG
    assert "ascending" in amgh.amgh_last_error()


def test_bench_sweep_work_counts(amgh):
    """The bench's FP64 view counts the finest colour sweep's work from the stars (columns of G),
    the star colours and A's row lengths; its vectorised count equals a plain loop over the stars
    of each colour step (0..C-1, C-2..0)."""
    import bench
    p = W.make_config("hex8_unit")
    h = amgh.amgh_setup_host_structure(p["A"], p["G"])
    colour = amgh.amgh_level_structure(h, 0)["colour"]
    amgh.amgh_destroy(h)
    by, fl = bench.finest_sweep_work(p["A"], p["G"], colour, 8, 8)
    Gc = p["G"].tocsc()
    rowlen = np.diff(p["A"].indptr)
    C = int(colour.max()) + 1
    seq = list(range(C)) + list(range(C - 2, -1, -1))
    by2 = fl2 = 0
    for c in seq:
        for j in np.flatnonzero(colour == c):
            rows = Gc.indices[Gc.indptr[j]:Gc.indptr[j + 1]]
            b = len(rows)
            for e in rows:
                by2 += rowlen[e] * 12 + b * 8 + 3 * 8
                fl2 += 2 * rowlen[e] + 2 * b + 2
    assert by == by2 and fl == fl2


def test_host_structure_matches_oracle_golden_at_bench_size(amgh):
    """Level 0 of the benchmark's workload (64^3 checkerboard): the library's host graph steps
    against the oracle's stored structure digests (tests/golden/hex64_checker.json, written by
    tests/golden/make_oracle_goldens.py from the oracle alone)."""
    import hashlib
    import json
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "hex64_checker.json")))
    d = gold["levels"][0]["digests"]

    def digest(arr, dtype):
        return hashlib.sha256(np.ascontiguousarray(np.asarray(arr), dtype=np.dtype(dtype).newbyteorder("<"))
                              .tobytes()).hexdigest()

    p = W.make_config("hex64_checker")
    h = amgh.amgh_setup_host_structure(p["A"], p["G"])
    s = amgh.amgh_level_structure(h, 0)
    assert digest(s["cf_state"], "i1") == d["cf_state"]
    assert digest(s["edges"].astype(np.int64), "i4") == d["edges"]
    assert digest(s["coarse_nodes"], "i4") == d["coarse_nodes"]
    assert digest(s["patch_ptr"], "i4") == d["patch_ptr"]
    assert digest(s["patch_idx"], "i4") == d["patch_idx"]
    assert digest(s["colour"], "i4") == d["colour"]


@pytest.mark.parametrize("n,geometric", [(8, False), (8, True), (16, False), (16, True)])
def test_refinement_structure_matches_oracle(amgh, n, geometric):
    """Section 3's refinement pairs ("Ref") and the geometric interpolation's supports ("Geo")
    from the library's host code against the oracle's: coarse edges with signs and end nodes,
    coarse nodes, patches (Geo: its supports), colours and the P pattern, bit for bit."""
    p = W.make_config("hex16_checker") if n == 16 else W.hex_problem(8, W.fields.checkerboard(8, 4), 1e-2)
    kw = dict(coarsening=amgh.AMGH_COARSEN_REFINEMENT, mesh_n=n)
    if geometric:
        kw["interp"] = amgh.AMGH_INTERP_GEOMETRIC
    h = amgh.amgh_setup_host_structure(p["A"], p["G"], **kw)
    s = amgh.amgh_level_structure(h, 0)
    cz = O.coarsen(p["A"], p["G"], splitting="refinement", mesh_n=n, interp="geometric" if geometric else "local")
    edges = np.array([[e[0], int(e[1]), e[2], int(e[3]), e[4], e[5], e[6]] for e in cz["edges"]], np.int64)
    np.testing.assert_array_equal(s["edges"].astype(np.int64), edges)
    np.testing.assert_array_equal(s["coarse_nodes"], cz["coarse_nodes"])
    np.testing.assert_array_equal(s["patch_idx"], np.concatenate(cz["patches"]))
    np.testing.assert_array_equal(s["colour"], O.colour_stars(p["A"], p["G"]))
    P = amgh.amgh_level_matrix(h, 0, 1)
    np.testing.assert_array_equal(P.indptr, cz["P"].indptr)
    np.testing.assert_array_equal(P.indices, cz["P"].indices)


def test_refinement_rejects_bad_meshes(amgh):
    p = W.hex_problem(8, 1.0, 1.0)
    with pytest.raises(amgh.AmghError) as e:
        amgh.amgh_setup_host_structure(p["A"], p["G"], coarsening=amgh.AMGH_COARSEN_REFINEMENT, mesh_n=7)
    assert e.value.status == amgh.AMGH_ERR_INVALID_ARG
    with pytest.raises(amgh.AmghError) as e:
        amgh.amgh_setup_host_structure(p["A"], p["G"], coarsening=amgh.AMGH_COARSEN_REFINEMENT, mesh_n=10)
    assert e.value.status == amgh.AMGH_ERR_INVALID_ARG
    with pytest.raises(amgh.AmghError) as e:
        amgh.amgh_setup_host_structure(p["A"], p["G"], interp=amgh.AMGH_INTERP_GEOMETRIC)
    assert e.value.status == amgh.AMGH_ERR_INVALID_ARG


@pytest.mark.parametrize("case", ["hex8_unit", "hex12_lognormal", "tri16", "hex8_ref", "hex16_checker"])
def test_commuting_nodal_interpolation_matches_oracle(amgh, case):
    """The nodal interpolation P_n of the commuting correction (reading R10) from the library's
    host code against the oracle's: pattern bit for bit, values to 1e-15 (the library sums a
    layer's neighbours, then divides; the oracle scales, then sums); on the hex refinement it is
    the trilinear interpolation the oracle's pin fixes."""
    kw, okw = {}, {}
    if case == "hex8_unit":
        p = W.make_config("hex8_unit")
    elif case == "hex12_lognormal":
        p = W.hex_problem(12, W.fields.log_uniform(12, 3, lo=-2, hi=2), 0.1)
    elif case == "tri16":
        p = W.tri_problem(16, 1.0, 0.01)
    elif case == "hex8_ref":
        p = W.hex_problem(8, 1.0, 1.0)
        kw = dict(coarsening=amgh.AMGH_COARSEN_REFINEMENT, mesh_n=8)
        okw = dict(splitting="refinement", mesh_n=8)
    else:
        p = W.make_config("hex16_checker")
    h = amgh.amgh_setup_host_structure(p["A"], p["G"], interp=amgh.AMGH_INTERP_CONSTRAINED, **kw)
    Pn = amgh.amgh_level_matrix(h, 0, 4)
    cz = O.coarsen(p["A"], p["G"], interp="constrained", **okw)
    m = p["G"].shape[1]
    want = sp.csr_matrix(cz["Pn"][:m])
    want.sort_indices()
    want.eliminate_zeros()
    assert Pn.shape == want.shape
    np.testing.assert_array_equal(Pn.indptr, want.indptr)
    np.testing.assert_array_equal(Pn.indices, want.indices)
    np.testing.assert_allclose(Pn.data, want.data, rtol=1e-15, atol=0)
    # without the correction there is no P_n to read
    h0 = amgh.amgh_setup_host_structure(p["A"], p["G"], **kw)
    with pytest.raises(amgh.AmghError) as e:
        amgh.amgh_level_matrix(h0, 0, 4)
    assert e.value.status == amgh.AMGH_ERR_INVALID_ARG
