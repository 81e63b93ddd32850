"""Failure detection without a GPU fault: the device-side bounded waits of the cooperative smoother
sweeps give up, raise the error flag and return, and the context stays usable afterwards."""
import numpy as np
import pytest

import workloads as W

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


def test_bounded_wait_gives_up_and_reports(amgh):
    st, sec = amgh.amgh_selftest_wait_timeout()
    print("grid barrier that cannot complete: status %d after %.2f s" % (st, sec))
    assert st == amgh.AMGH_ERR_TIMEOUT
    assert sec < 10.0
    # the context is still usable: a full setup and solve succeed afterwards
    p = W.make_config("hex8_unit")
    h = amgh.amgh_setup(p["A"], p["G"])
    x = np.zeros(p["ndof"])
    it, rel, ok = amgh.amgh_pcg_solve(h, p["f"], x, 1e-8, 100)
    assert ok and rel <= 1e-8
