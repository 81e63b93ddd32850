"""The allocation-free PCG entry point (for callers that cannot allocate device memory when they
solve, e.g. under a caching allocator that holds nearly all device memory) must give what
amgh_pcg_solve gives, call after call, with its Krylov buffers in the library's fixed device
array, and leave the device's free memory unchanged.  Kept in its own file, collected last."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def amgh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2602_23613_gb300 import build, amgh as mod
    build.build()
    mod.load()
    return mod


@pytest.mark.parametrize("prec,case", [("f64", "hex16_checker"), ("f32", "hex8_unit")])
def test_noalloc_matches_pcg_twice(amgh, prec, case):
    import torch
    code = {"f64": amgh.AMGH_F64, "f32": amgh.AMGH_F32}[prec]
    p = W.make_config(case)
    h = amgh.amgh_setup(p["A"], p["G"], precision=code)
    f = torch.tensor(p["f"], device="cuda")
    ref = torch.zeros_like(f)
    it_ref, rel_ref, ok_ref = amgh.amgh_pcg_solve(h, f, ref, 1e-8, 300)
    assert ok_ref
    scale = float(ref.abs().max())
    xs = [torch.zeros_like(f) for _ in range(2)]
    torch.cuda.synchronize()
    for call in range(2):                      # the shared array keeps the last call's contents
        x = xs[call]
        free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        it, rel, ok = amgh.amgh_pcg_solve_noalloc(h, f, x, 1e-8, 300)
        torch.cuda.synchronize()
        if call == 1:                          # the first call may load the module's device array
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_reserved() == reserved0
        assert ok and it == it_ref, (call, it, it_ref)
        assert abs(rel - rel_ref) <= TOL * max(rel_ref, 1e-300) + 1e-300 or rel == rel_ref
        assert float((x - ref).abs().max()) <= TOL * scale, call


def test_noalloc_rejects_large_and_host_inputs(amgh):
    import torch
    p = W.hex_problem(48, 1.0, 1.0)                 # 3*48*47^2 = 318,096 rows > 262,144
    h = amgh.amgh_setup(p["A"], p["G"])
    f = torch.ones(p["ndof"], dtype=torch.float64, device="cuda")
    x = torch.zeros_like(f)
    with pytest.raises(amgh.AmghError) as e:
        amgh.amgh_pcg_solve_noalloc(h, f, x, 1e-8, 10)
    assert e.value.status == amgh.AMGH_ERR_INVALID_ARG
    assert "at most 262144" in str(e.value)
    q = W.make_config("hex8_unit")
    hq = amgh.amgh_setup(q["A"], q["G"])
    xh = np.zeros(q["ndof"])
    with pytest.raises(amgh.AmghError) as e:
        amgh.amgh_pcg_solve_noalloc(hq, q["f"], xh, 1e-8, 10)
    assert e.value.status == amgh.AMGH_ERR_INVALID_ARG
