"""Failure detection without a GPU fault: every spin-wait of the library's
kernels is bounded; a wait that runs out records the give-up in a device
status word, the kernel returns, the host call reports CC3_ERR_TIMEOUT and the
CUDA context stays usable.  The wait is made to run out on an mbarrier that
nothing arrives on (a 1 ms limit, nothing else in flight)."""
import time

import numpy as np
import pytest

from cc3_inputs import make_inputs


def test_wait_limit_out_of_range_is_rejected_on_the_host():
    import paper_2007_01088_gb300 as g
    for bad in (0.0, -1.0, 2.0, float("nan")):
        assert g.cc3_debug_wait_timeout(bad) == g.CC3_ERR_ARG


@pytest.mark.gpu
def test_bounded_wait_times_out_and_the_context_survives():
    import oracle
    import paper_2007_01088_gb300 as g
    t0 = time.perf_counter()
    assert g.cc3_debug_wait_timeout(1e-3) == g.CC3_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert "gave up" in g.cc3_last_error()
    assert g.cc3_debug_wait_timeout(2e-3) == g.CC3_ERR_TIMEOUT  # and again
    # the device context is intact: a residual on both paths still matches
    inp = make_inputs(3, 20, seed=9)
    ref = oracle.omega_inputs(inp)
    ctx = g.Context(inp)
    for prec in (g.CC3_FP64, g.CC3_SPLIT_BF16):
        o1, o2, e = ctx.omega(prec)
        assert np.abs(o2 - ref["omega2"]).max() <= 1e-9
