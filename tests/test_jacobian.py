"""Right CC3 Jacobian transformation (triples part) through the C ABI against
the oracle (eq. "jcc3" with the Algorithm 2 intermediates on the GPU side, the
direct tau~3 . g^ contractions on the oracle side).

FP64 path: 1e-11 relative to the largest element of the reference, elementwise
(a few hundred FP64 roundings in the longest sums, well below that bound).
Split path: the residual's absolute targets (1e-9) scaled by the size of the
transformed vector."""
import numpy as np
import pytest

import oracle
from cc3_inputs import make_inputs, make_trial_vectors, unique_triples

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2007_01088_gb300 as g
    return g


def _close(x, ref, rel):
    scale = max(np.abs(ref).max(), 1e-300)
    return np.abs(np.asarray(x) - ref).max() <= rel * scale


@pytest.mark.parametrize("no,nv", [(3, 9), (4, 20), (2, 17), (5, 33)])
def test_jacobian_fp64_matches_oracle(g, no, nv):
    inp = make_inputs(no, nv, seed=100 + no * nv)
    R1, R2 = make_trial_vectors(no, nv, 2, seed=no + nv)
    w = [0.25, 0.0]
    ref = oracle.jacobian(inp, R1, R2, w)
    ctx = g.Context(inp)
    r1, r2 = ctx.jacobian(R1, R2, w, g.CC3_FP64)
    assert _close(r1, ref["rho1"], 1e-11)
    assert _close(r2, ref["rho2"], 1e-11)
    # second call reuses the cached Algorithm 2 intermediates
    r1b, r2b = ctx.jacobian(R1[1:], R2[1:], w[1:], g.CC3_FP64)
    assert _close(r1b[0], ref["rho1"][1], 1e-11)
    assert _close(r2b[0], ref["rho2"][1], 1e-11)
    c = ctx.counters()
    assert c["launches"] > 0 and c["nominal_flop"] > 0


def test_jacobian_fp64_device_pointers(g):
    import torch
    no, nv = 4, 18
    inp = make_inputs(no, nv, seed=7)
    R1, R2 = make_trial_vectors(no, nv, 3, seed=3)
    w = [0.1, -0.05, 0.3]
    ref = oracle.jacobian(inp, R1, R2, w)
    ctx = g.Context(inp, device=True)
    r1, r2 = ctx.jacobian(torch.from_numpy(R1).cuda(), torch.from_numpy(R2).cuda(), w,
                          g.CC3_FP64)
    torch.cuda.synchronize()
    assert _close(r1.cpu().numpy(), ref["rho1"], 1e-11)
    assert _close(r2.cpu().numpy(), ref["rho2"], 1e-11)


def test_jacobian_fp64_triple_subset_and_cache_invalidation(g):
    no, nv = 5, 16
    inp = make_inputs(no, nv, seed=11)
    R1, R2 = make_trial_vectors(no, nv, 1, seed=5)
    ctx = g.Context(inp)
    ctx.jacobian(R1, R2, [0.2], g.CC3_FP64)  # fills the cache for all triples
    tri = [t[:3] for t in unique_triples(no)][::3]
    ctx.set_triples(tri)
    r1, r2 = ctx.jacobian(R1, R2, [0.2], g.CC3_FP64)
    ref = oracle.jacobian(inp, R1, R2, [0.2], triples=tri)
    assert _close(r1, ref["rho1"], 1e-11)
    assert _close(r2, ref["rho2"], 1e-11)


def test_jacobian_on_t2_gives_residual(g):
    # R = (0, t2) at w = 0 turns R3 into tau3 itself: rho = the residual's
    # contractions of tau~3 with the plain integrals (= Omega)
    no, nv = 4, 15
    inp = make_inputs(no, nv, seed=21)
    ctx = g.Context(inp)
    r1, r2 = ctx.jacobian(np.zeros((1, no, nv)), np.ascontiguousarray(inp.t2[None]), [0.0],
                          g.CC3_FP64)
    o1, o2, _ = ctx.omega(g.CC3_FP64)
    assert _close(r1[0], o1, 1e-11)
    assert _close(r2[0], o2, 1e-11)


def test_jacobian_needs_cholesky_vectors(g):
    inp = make_inputs(3, 8, seed=1, keep_chol=False)
    ctx = g.Context(inp)
    R1, R2 = make_trial_vectors(3, 8, 1)
    with pytest.raises(g.CC3Error) as e:
        ctx.jacobian(R1, R2, [0.0], g.CC3_FP64)
    assert e.value.status == g.CC3_ERR_ARG


# split path: Omega-scale absolute targets (the trial vectors are normalised)
SPLIT_TOL = 1e-9


@pytest.mark.parametrize("no,nv", [(3, 9), (4, 20), (5, 33), (3, 40)])
def test_jacobian_split_matches_oracle(g, no, nv):
    inp = make_inputs(no, nv, seed=300 + no * nv)
    R1, R2 = make_trial_vectors(no, nv, 3, seed=no * nv)
    w = [0.25, 0.0, -0.1]
    ref = oracle.jacobian(inp, R1, R2, w)
    ctx = g.Context(inp)
    r1, r2 = ctx.jacobian(R1, R2, w, g.CC3_SPLIT_BF16)
    assert np.abs(r1 - ref["rho1"]).max() <= SPLIT_TOL
    assert np.abs(r2 - ref["rho2"]).max() <= SPLIT_TOL
    c = ctx.counters()
    assert c["slices"] == 6 and c["executed_flop"] > 0


def test_jacobian_split_and_fp64_share_the_context(g):
    no, nv = 4, 24
    inp = make_inputs(no, nv, seed=17)
    R1, R2 = make_trial_vectors(no, nv, 2, seed=2)
    w = [0.2, 0.05]
    ref = oracle.jacobian(inp, R1, R2, w)
    ctx = g.Context(inp)
    s1, s2 = ctx.jacobian(R1, R2, w, g.CC3_SPLIT_BF16)  # builds the Z~ cache in split
    f1, f2 = ctx.jacobian(R1, R2, w, g.CC3_FP64)        # rebuilds it in FP64
    assert _close(f2, ref["rho2"], 1e-11) and _close(f1, ref["rho1"], 1e-11)
    t1, t2 = ctx.jacobian(R1, R2, w, g.CC3_SPLIT_BF16)  # reuses the FP64 cache
    for x, y in ((s1, ref["rho1"]), (s2, ref["rho2"]), (t1, ref["rho1"]), (t2, ref["rho2"])):
        assert np.abs(x - y).max() <= SPLIT_TOL
