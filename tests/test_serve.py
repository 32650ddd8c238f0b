"""Serving loop (continuous batching) through the C ABI: each result in a mix
of concurrently admitted requests equals the same request evaluated alone,
admission respects the HBM budget, failures stay with their request, and
queued requests can be cancelled."""
import numpy as np
import pytest

from cc3_inputs import make_inputs, make_trial_vectors
from split_tol import energy_close, split_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2007_01088_gb300 as g
    return g


def _rel(x, ref):
    return np.abs(np.asarray(x) - ref).max() / max(np.abs(ref).max(), 1e-300)


# (kind, prec, no, nv, nvec)
MIX = [("omega", "fp64", 4, 30, 0), ("omega", "split", 5, 40, 0), ("jac", "fp64", 3, 20, 2),
       ("omega", "fp64", 6, 24, 0), ("omega", "split", 3, 17, 0), ("jac", "fp64", 4, 25, 1),
       ("jac", "split", 4, 22, 2)]


def _alone(g, inp, kind, prec, R=None):
    ctx = g.Context(inp)
    try:
        if kind == "omega":
            return ctx.omega(prec)
        return ctx.jacobian(R[0], R[1], R[2], prec)
    finally:
        ctx.close()


def test_mix_equals_alone(g):
    probs = []
    for n, (kind, p, no, nv, nvec) in enumerate(MIX):
        prec = g.CC3_FP64 if p == "fp64" else g.CC3_SPLIT_BF16
        inp = make_inputs(no, nv, seed=50 + n)
        R = None
        if kind == "jac":
            R1, R2 = make_trial_vectors(no, nv, nvec, seed=n)
            R = (R1, R2, np.linspace(0.0, 0.3, nvec))
        probs.append((kind, prec, inp, R))
    alone = [_alone(g, inp, kind, prec, R) for kind, prec, inp, R in probs]
    srv = g.Server(max_slots=3)
    try:
        fps, tickets = [], []
        for kind, prec, inp, R in probs:
            if kind == "omega":
                fps.append(srv.footprint(0, prec, inp))
                tickets.append(srv.submit_omega(inp, prec))
            else:
                fps.append(srv.footprint(1, prec, inp, len(R[2]), R[2], R[0], R[1]))
                tickets.append(srv.submit_jacobian(inp, R[0], R[1], R[2], prec))
        for (kind, prec, inp, R), t, ref in zip(probs, tickets, alone):
            st, out = srv.wait(t)
            assert st == g.CC3_OK
            if kind == "omega" and prec == g.CC3_FP64:
                assert _rel(out[0], ref[0]) <= 1e-12 and _rel(out[1], ref[1]) <= 1e-12
                assert abs(out[2][0] - ref[2][0]) <= 1e-12 * abs(ref[2][0])
            elif kind == "omega":
                assert split_close(out[0], ref[0]) and split_close(out[1], ref[1])
                assert energy_close(out[2][0], ref[2][0])
            elif prec == g.CC3_FP64:
                assert _rel(out[0], ref[0]) <= 1e-11 and _rel(out[1], ref[1]) <= 1e-11
            else:
                assert split_close(out[0], ref[0]) and split_close(out[1], ref[1])
        s = srv.stats()
        assert s["completed"] == len(MIX) and s["admitted"] == len(MIX)
        assert s["rejected"] == 0 and s["cancelled"] == 0
        assert 0 < s["p50_ms"] <= s["p99_ms"]
        assert s["nominal_flop"] > 0 and s["hbm_in_use"] == 0
        # several requests were resident at once (continuous batching)
        assert s["hbm_peak"] > max(fps)
    finally:
        srv.stop()


def test_admission_respects_budget_and_rejects_oversize(g):
    small = [make_inputs(4, 20 + 2 * n, seed=n) for n in range(4)]
    srv0 = g.Server(max_slots=1)
    fp = max(srv0.footprint(0, g.CC3_FP64, x) for x in small)
    big = make_inputs(8, 90, seed=3)
    fp_big = srv0.footprint(0, g.CC3_FP64, big)
    srv0.stop()
    assert fp_big > 1.5 * fp
    budget = int(1.5 * fp)  # one request at a time
    srv = g.Server(hbm_budget_bytes=budget, max_slots=4)
    try:
        ts = [srv.submit_omega(x) for x in small]
        with pytest.raises(g.CC3Error) as e:
            srv.submit_omega(big)
        assert e.value.status == g.CC3_ERR_BUSY
        for t in ts:
            assert srv.wait(t)[0] == g.CC3_OK
        s = srv.stats()
        assert s["hbm_peak"] <= budget and s["rejected"] == 1 and s["completed"] == 4
    finally:
        srv.stop()


def test_failed_request_is_isolated(g):
    good = make_inputs(4, 18, seed=1)
    bad = make_inputs(4, 18, seed=2)
    bad.eps_v = -np.abs(bad.eps_v)  # every denominator eps^{abc}_{ijk} <= 0
    srv = g.Server(max_slots=2)
    try:
        t1 = srv.submit_omega(good)
        t2 = srv.submit_omega(bad)
        t3 = srv.submit_omega(good)
        assert srv.wait(t2)[0] == g.CC3_ERR_DENOM
        st1, o1 = srv.wait(t1)
        st3, o3 = srv.wait(t3)
        assert st1 == g.CC3_OK and st3 == g.CC3_OK
        assert _rel(o1[1], o3[1]) <= 1e-12
    finally:
        srv.stop()


def test_cancel_queued_and_wait_timeout(g):
    a = make_inputs(8, 80, seed=4)
    b = make_inputs(3, 12, seed=5)
    srv = g.Server(max_slots=1)
    try:
        ta = srv.submit_omega(a)
        tb = srv.submit_omega(b)
        srv.cancel(tb)
        st, _ = srv.wait(ta, 0.0)
        assert st in (g.CC3_ERR_TIMEOUT, g.CC3_OK)
        if st == g.CC3_ERR_TIMEOUT:
            assert srv.wait(ta)[0] == g.CC3_OK
        assert srv.wait(tb)[0] == g.CC3_ERR_CANCELLED
        with pytest.raises(g.CC3Error):
            srv.wait(tb)  # ticket released
        assert srv.stats()["cancelled"] == 1
    finally:
        srv.stop()


def test_footprint_bounds_device_memory(g):
    import torch
    torch.cuda.init()
    srv = g.Server(max_slots=1)
    try:
        for prec, no, nv in [(g.CC3_FP64, 6, 60), (g.CC3_SPLIT_BF16, 6, 60),
                             (g.CC3_FP64, 10, 48)]:
            inp = make_inputs(no, nv, seed=9)
            fp = srv.footprint(0, prec, inp)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            ctx = g.Context(inp)
            ctx.omega(prec)
            used = free0 - torch.cuda.mem_get_info()[0]
            ctx.close()
            assert used <= fp, (prec, no, nv, used, fp)
    finally:
        srv.stop()


def test_deterministic_requests_are_bitwise_equal_alone_and_in_the_mix(g):
    probs = [(make_inputs(4 + n, 20 + 6 * n, seed=80 + n),
              g.CC3_SPLIT_BF16 if n % 2 else g.CC3_FP64) for n in range(5)]
    alone = []
    for inp, prec in probs:
        ctx = g.Context(inp, flags=g.CC3_DETERMINISTIC)
        alone.append(ctx.omega(prec))
        ctx.close()
    srv = g.Server(max_slots=3)
    try:
        ts = [srv.submit_omega(inp, prec, flags=g.CC3_DETERMINISTIC) for inp, prec in probs]
        for t, ref in zip(ts, alone):
            st, out = srv.wait(t)
            assert st == g.CC3_OK
            for x, y in zip(out, ref):
                assert np.array_equal(x, y)
    finally:
        srv.stop()
