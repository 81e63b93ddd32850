"""Write the oracle's reference values for a named workload to tests/golden/<name>.json.

Calls only the CPU oracle (oracle/amg.py) and the seeded input generators (workloads/).  The
library is never imported here: every stored value is the oracle's.

Stored per level l of the oracle hierarchy (default parameters: coarse size 100, p_max 128, ring 1):
  * n, nnz, and SHA-256 digests of the structure (little-endian bytes): the C/F state of the
    augmented nodes (int8, 1 = C incl. boundary nodes, 2 = F), the coarse edges
    (int32 rows dof1, s1, dof2, s2, i, k, j), the coarse nodes, the patch pointers and indices,
    the star colours, and the CSR patterns (row pointers, column indices) of A_l and P_l;
  * the values of A_l and P_l on a seeded sample of rows;
  * the largest condition numbers of the star blocks and the patch blocks (the parity tests'
    per-level tolerance is max(1e-12, 8 eps kappa)).
And for the whole hierarchy: one V-cycle of a seeded vector (norms and sampled entries), and the
PCG solve of the workload's right-hand side to 1e-8 (iterations, residual history, energy f.x,
sampled entries of x).

Usage: python tests/golden/make_oracle_goldens.py hex64_checker   (about an hour on one core)
       python tests/golden/make_oracle_goldens.py hex64_checker constrained
           (the local extension corrected to commute, readings R10-R11; written to
           tests/golden/hex64_checker_constrained.json)
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads as W          # noqa: E402
from oracle import amg as O    # noqa: E402


def digest(arr, dtype):
    return hashlib.sha256(np.ascontiguousarray(np.asarray(arr), dtype=np.dtype(dtype).newbyteorder("<"))
                          .tobytes()).hexdigest()


def structure_digests(L):
    A = L["A"]
    out = dict(A_indptr=digest(A.indptr, "i4"), A_indices=digest(A.indices, "i4"),
               colour=digest(L["colour"], "i4"))
    cz = L.get("coarsening")
    if cz is None:
        return out
    state = np.full(cz["Gt"].shape[1], 2, np.int8)
    state[cz["cG"]] = 1
    state[cz["B"]] = 1
    edges = np.array([[e[0], int(e[1]), e[2], int(e[3]), e[4], e[5], e[6]] for e in cz["edges"]], np.int64)
    pptr = np.concatenate([[0], np.cumsum([len(x) for x in cz["patches"]])])
    P = cz["P"]
    out.update(cf_state=digest(state, "i1"), edges=digest(edges, "i4"), coarse_nodes=digest(cz["coarse_nodes"], "i4"),
               patch_ptr=digest(pptr, "i4"), patch_idx=digest(np.concatenate(cz["patches"]), "i4"),
               P_indptr=digest(P.indptr, "i4"), P_indices=digest(P.indices, "i4"))
    return out


def sampled_rows(M, rows):
    return dict(rows=[int(r) for r in rows],
                values=[[float(v) for v in M.data[M.indptr[r]:M.indptr[r + 1]]] for r in rows])


def max_cond(A, blocks):
    """Largest 2-norm condition number over the dense blocks A[b][:, b], batched by block size."""
    by_size = {}
    for b in blocks:
        if len(b):
            by_size.setdefault(len(b), []).append(b)
    worst = 1.0
    Ad = A.tocsr()
    for m, bs in by_size.items():
        for s in range(0, len(bs), 4096):
            stack = np.stack([Ad[b][:, b].toarray() for b in bs[s:s + 4096]])
            worst = max(worst, float(np.linalg.cond(stack).max()))
    return worst


def main(name, interp="local", out_path=None):
    t0 = time.time()
    p = W.make_config(name)
    print("inputs %.1f s" % (time.time() - t0), flush=True)
    t = time.time()
    H = O.setup(p["A"], p["G"], interp=interp)
    t_setup = time.time() - t
    print("oracle setup %.1f s, levels %s" % (t_setup, [L["A"].shape[0] for L in H]), flush=True)
    rng = np.random.default_rng(20260101)
    levels = []
    for l, L in enumerate(H):
        A = L["A"]
        n = A.shape[0]
        nrow = 32 if n > 50000 else 8
        rows = np.sort(rng.choice(n, min(nrow, n), replace=False))
        lev = dict(n=int(n), nnz=int(A.nnz), ncolours=int(L["ncolours"]), digests=structure_digests(L),
                   A_rows=sampled_rows(A, rows), kappa_star=max_cond(A, L["stars"]))
        cz = L.get("coarsening")
        if cz is not None:
            P = cz["P"]
            prow = np.sort(rng.choice(n, min(nrow, n), replace=False))
            lev.update(nc=int(P.shape[1]), P_nnz=int(P.nnz), P_rows=sampled_rows(P, prow),
                       kappa_patch=max_cond(A, cz["patches"]))
        levels.append(lev)
        print("level %d: n %d, digests and kappas done (%.1f s)" % (l, n, time.time() - t0), flush=True)
    n0 = H[0]["A"].shape[0]
    idx = np.sort(rng.choice(n0, min(4096, n0), replace=False))
    r = W.uniform("probe", 100, n0)
    t = time.time()
    z = O.vcycle(H, r)
    t_vc = time.time() - t
    print("V-cycle %.1f s" % t_vc, flush=True)
    vcyc = dict(probe_stream="probe", probe_seed=100, inf_norm=float(np.abs(z).max()),
                two_norm=float(np.linalg.norm(z)), idx=[int(i) for i in idx], values=[float(z[i]) for i in idx])
    t = time.time()
    x, it, hist = O.pcg(H, p["f"], tol=1e-8, maxit=1000)
    t_pcg = time.time() - t
    print("PCG %d iterations, %.1f s" % (it, t_pcg), flush=True)
    pcg = dict(tol=1e-8, iterations=int(it), relres=[float(h / hist[0]) for h in hist],
               energy=float(p["f"] @ x), inf_norm=float(np.abs(x).max()),
               idx=[int(i) for i in idx[:1024]], values=[float(x[i]) for i in idx[:1024]])
    out = dict(workload=name, description=W.describe(name)[0], generator="tests/golden/make_oracle_goldens.py",
               params=dict(coarse_size=100, p_max=128, ring=1, strength="classical", theta=0.25, interp=interp),
               oracle_seconds=dict(setup=t_setup, vcycle=t_vc, pcg=t_pcg),
               levels=levels, vcycle=vcyc, pcg=pcg)
    out_path = out_path or os.path.join(HERE, name + ("" if interp == "local" else "_" + interp) + ".json")
    with open(out_path, "w") as fh:
        json.dump(out, fh, indent=None, separators=(",", ":"))
        fh.write("\n")
    print("wrote %s (%.1f s in all)" % (out_path, time.time() - t0), flush=True)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "hex64_checker", sys.argv[2] if len(sys.argv) > 2 else "local",
         sys.argv[3] if len(sys.argv) > 3 else None)
