"""Every launch mode of the Schwarz colour sweep gives the oracle's smoothing steps and V-cycle.

The autotuner picks one mode per level by timing, so the parity tests only see the modes it
picked; here each mode is forced (AMGH_SMOOTHER_MODE, read at setup) on a hierarchy whose levels
support it, and every level's pre-/post-step and the whole V-cycle are compared with the oracle
within the kappa-derived tolerances of the parity tests.  Modes a level cannot run (too many
chunks for a cluster, too large a level for one CTA, ...) fall back to per-colour launches there,
and amgh_info reports which mode each level got."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import amg as O

from test_gpu_parity import level_tols, rel, vcycle_tol

pytestmark = pytest.mark.gpu

MODES = ["colour", "pdl", "stream1", "stream2", "fused", "persistent", "staged", "cluster", "cluster2", "resident",
         "pipeline"]
CODE = {"colour": 0, "fused": 1, "persistent": 2, "staged": 3, "stream1": 4, "stream2": 4, "cluster": 5, "pdl": 6,
        "cluster2": 7, "resident": 8, "pipeline": 9}


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
    p = W.make_config("hex16_checker")
    H = O.setup(p["A"], p["G"], coarse_size=100)
    return p, H, level_tols(H)


@pytest.mark.parametrize("mode", MODES)
def test_forced_mode_matches_oracle(amgh, problem, mode):
    import torch
    p, H, tols = problem
    old = os.environ.get("AMGH_SMOOTHER_MODE")
    os.environ["AMGH_SMOOTHER_MODE"] = mode
    try:
        h = amgh.amgh_setup(p["A"], p["G"], dense_tail=0)
    finally:
        if old is None:
            del os.environ["AMGH_SMOOTHER_MODE"]
        else:
            os.environ["AMGH_SMOOTHER_MODE"] = old
    info = amgh.amgh_info(h)
    used = [info["fused"][l] for l in range(info["levels"] - 1)]
    print("forced %s: level modes %s" % (mode, used))
    assert CODE[mode] in used or mode in ("fused", "cluster", "cluster2", "persistent", "staged", "resident",
                                          "pipeline")
    for l in range(info["levels"] - 1):
        L = H[l]
        n = L["A"].shape[0]
        f = W.uniform("probe", 40 + l, n)
        x = W.uniform("probe", 60 + l, n)
        fd, xd = torch.tensor(f, device="cuda"), torch.tensor(x, device="cuda")
        y = torch.zeros_like(fd)
        amgh.amgh_level_apply(h, l, 2, fd, xd, y)
        assert rel(y.cpu().numpy(), O.smooth_pre(L, f, x.copy())) < tols[l]["smooth"], (mode, l, "pre-step")
        amgh.amgh_level_apply(h, l, 3, fd, xd, y)
        assert rel(y.cpu().numpy(), O.smooth_post(L, f, x.copy())) < tols[l]["smooth"], (mode, l, "post-step")
    r = torch.tensor(W.uniform("probe", 7, p["ndof"]), device="cuda")
    z = torch.zeros_like(r)
    amgh.amgh_vcycle(h, r, z)
    assert rel(z.cpu().numpy(), O.vcycle(H, r.cpu().numpy())) < vcycle_tol(tols), mode


RESIDENT = ["resident-%dx%d-L%d" % (c, g, l) for c in (16, 8) for g in (1, 2) for l in (4, 8, 16, 32)]
PIPELINE = ["pipeline-%dx%d-L%d" % (c, g, l) for c in (152, 38) for g in (1, 2) for l in (4, 32)]


@pytest.mark.parametrize("shape", RESIDENT + PIPELINE)
def test_resident_shape_matches_oracle(amgh, problem, shape):
    """Every shape of the resident sweep (cluster size, chunk groups per CTA, lanes per row) and of
    its grid form (grid size, chunk groups, lanes): with 4 lanes and two groups the rows of levels
    1-2 (up to 108 entries) run past the 16 prefetched entries per lane, and the finest level's
    colours have more chunks than the cluster has groups."""
    import torch
    p, H, tols = problem
    old = os.environ.get("AMGH_SMOOTHER_MODE")
    os.environ["AMGH_SMOOTHER_MODE"] = shape
    try:
        h = amgh.amgh_setup(p["A"], p["G"], dense_tail=0)
    finally:
        if old is None:
            del os.environ["AMGH_SMOOTHER_MODE"]
        else:
            os.environ["AMGH_SMOOTHER_MODE"] = old
    info = amgh.amgh_info(h)
    used = [info["fused"][l] for l in range(info["levels"] - 1)]
    lanes = [info["lanes"][l] for l in range(info["levels"] - 1)]
    print("forced %s: level modes %s, lanes %s" % (shape, used, lanes))
    assert CODE[shape.split("-")[0]] in used
    for l in range(info["levels"] - 1):
        L = H[l]
        n = L["A"].shape[0]
        f = W.uniform("probe", 40 + l, n)
        x = W.uniform("probe", 60 + l, n)
        fd, xd = torch.tensor(f, device="cuda"), torch.tensor(x, device="cuda")
        y = torch.zeros_like(fd)
        amgh.amgh_level_apply(h, l, 2, fd, xd, y)
        assert rel(y.cpu().numpy(), O.smooth_pre(L, f, x.copy())) < tols[l]["smooth"], (shape, l, "pre-step")
        amgh.amgh_level_apply(h, l, 3, fd, xd, y)
        assert rel(y.cpu().numpy(), O.smooth_post(L, f, x.copy())) < tols[l]["smooth"], (shape, l, "post-step")
    r = torch.tensor(W.uniform("probe", 7, p["ndof"]), device="cuda")
    z = torch.zeros_like(r)
    amgh.amgh_vcycle(h, r, z)
    assert rel(z.cpu().numpy(), O.vcycle(H, r.cpu().numpy())) < vcycle_tol(tols), shape
