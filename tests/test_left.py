"""Left (transpose) CC3 Jacobian transformation through the C ABI against the
oracle (oracle.left_jacobian: the transpose-Jacobian paragraph of the paper's
"Implementation" and the L3 amplitudes of Algorithm 3, read as the exact
transpose of the right transformation).  FP64 path: 1e-11 relative to the
largest reference element, as the right Jacobian's tests.  The batched shape
(no = 20, nv = 200, naux = 660) is checked on a triple subset against the
matrix-product form of the oracle."""
import numpy as np
import pytest

import oracle
from cc3_inputs import config_inputs, make_inputs, make_trial_vectors, unique_triples
from split_tol import split_close, split_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2007_01088_gb300 as g
    return g


def _close(x, ref, rel):
    return np.abs(np.asarray(x) - ref).max() <= rel * max(np.abs(ref).max(), 1e-300)


def _left_vectors(no, nv, n, seed):
    rng = np.random.default_rng(seed)
    L2 = rng.normal(size=(n, no, no, nv, nv))
    return rng.normal(size=(n, no, nv)), 0.5 * (L2 + np.transpose(L2, (0, 2, 1, 4, 3)))


@pytest.mark.parametrize("no,nv", [(3, 9), (4, 20), (2, 17), (5, 33)])
def test_left_jacobian_matches_oracle(g, no, nv):
    inp = make_inputs(no, nv, seed=200 + no * nv)
    L1, L2 = _left_vectors(no, nv, 2, seed=no + nv)
    w = [0.25, 0.0]
    ref = oracle.left_jacobian(inp, L1, L2, w)
    ctx = g.Context(inp)
    s1, s2 = ctx.left_jacobian(L1, L2, w)
    assert _close(s1, ref["sigma1"], 1e-11)
    assert _close(s2, ref["sigma2"], 1e-11)
    c = ctx.counters()
    assert c["nominal_flop"] == 8 * nv ** 4 * (no ** 3 - no) * 2 and c["launches"] > 0
    # a second call reuses the cached Algorithm 2 intermediates
    t1, t2 = ctx.left_jacobian(L1[1:], L2[1:], w[1:])
    assert _close(t1[0], ref["sigma1"][1], 1e-11) and _close(t2[0], ref["sigma2"][1], 1e-11)


def test_left_and_right_transformations_are_transposes(g):
    no, nv = 4, 24
    inp = make_inputs(no, nv, seed=33)
    R1, R2 = make_trial_vectors(no, nv, 2, seed=4)
    L1, L2 = _left_vectors(no, nv, 2, seed=6)
    ctx = g.Context(inp)
    for w in (0.3, 0.0):
        r1, r2 = ctx.jacobian(R1, R2, [w, w], g.CC3_FP64)
        s1, s2 = ctx.left_jacobian(L1, L2, [w, w])
        for n in range(2):
            for m in range(2):
                a = np.sum(L1[n] * r1[m]) + np.sum(L2[n] * r2[m])
                b = np.sum(s1[n] * R1[m]) + np.sum(s2[n] * R2[m])
                assert abs(a - b) <= 1e-12 * (np.abs(L2[n]).sum() * np.abs(r2[m]).max()
                                              + np.abs(L1[n]).sum() * np.abs(r1[m]).max())


def test_left_jacobian_device_pointers_and_subset(g):
    import torch
    no, nv = 5, 16
    inp = make_inputs(no, nv, seed=41)
    L1, L2 = _left_vectors(no, nv, 1, seed=2)
    tri = [t[:3] for t in unique_triples(no)][1::3]
    ref = oracle.left_jacobian(inp, L1, L2, [0.15], triples=tri)
    ctx = g.Context(inp, device=True)
    ctx.set_triples(tri)
    s1, s2 = ctx.left_jacobian(torch.from_numpy(L1).cuda(), torch.from_numpy(L2).cuda(), [0.15])
    torch.cuda.synchronize()
    assert _close(s1.cpu().numpy(), ref["sigma1"], 1e-11)
    assert _close(s2.cpu().numpy(), ref["sigma2"], 1e-11)


def test_left_jacobian_refusals(g):
    no, nv = 3, 10
    inp = make_inputs(no, nv, seed=8)
    L1, L2 = _left_vectors(no, nv, 1, seed=1)
    ctx = g.Context(inp)
    with pytest.raises(g.CC3Error) as e:
        ctx.left_jacobian(L1, L2, [0.0], g.CC3_SPLIT_INT8)
    assert e.value.status == g.CC3_ERR_UNSUPPORTED
    w_bad = inp.eps_v[0] + inp.eps_v[1] + inp.eps_v[2] - inp.eps_o.sum() + 1e-8
    with pytest.raises(g.CC3Error) as e:
        ctx.left_jacobian(L1, L2, [w_bad])
    assert e.value.status == g.CC3_ERR_DENOM


def test_left_jacobian_batched_shape(g):
    from oracle import matrix_form as MF
    inp = config_inputs("cfg4_jacobian_no20_nv200")
    no, nv = inp.no, inp.nv
    L1, L2 = _left_vectors(no, nv, 3, seed=12)
    w = [0.25, 0.0, -0.1]
    tr = [t[:3] for t in unique_triples(no)]
    rng = np.random.default_rng(9)
    sel = [tr[i] for i in sorted(rng.choice(len(tr), size=2, replace=False))] + [(18, 18, 3)]
    ref = MF.left_jacobian(inp, L1, L2, w, triples=sel)
    ctx = g.Context(inp)
    ctx.set_triples(sel)
    s1, s2 = ctx.left_jacobian(L1, L2, w)
    assert _close(s1, ref["sigma1"], 1e-11)
    assert _close(s2, ref["sigma2"], 1e-11)


# ---- split (BF16 slice) path -------------------------------------------------------------
# Left vectors normalised like the trial vectors, so that the absolute targets
# of the split path apply as for rho.

@pytest.mark.parametrize("no,nv", [(3, 9), (4, 20), (2, 17), (5, 33)])
def test_split_left_jacobian_matches_oracle(g, no, nv):
    inp = make_inputs(no, nv, seed=500 + no * nv)
    L1, L2 = make_trial_vectors(no, nv, 2, seed=no + 3 * nv)
    w = [0.25, 0.0]
    ref = oracle.left_jacobian(inp, L1, L2, w)
    ctx = g.Context(inp)
    s1, s2 = ctx.left_jacobian(L1, L2, w, g.CC3_SPLIT_BF16)
    assert split_close(s1, ref["sigma1"]), split_err(s1, ref["sigma1"])
    assert split_close(s2, ref["sigma2"]), split_err(s2, ref["sigma2"])
    c = ctx.counters()
    assert c["slices"] == 6 and c["launches"] > 0
    # FP64 after split on the same context (shared Algorithm 2 cache)
    f1, f2 = ctx.left_jacobian(L1, L2, w)
    assert _close(f1, ref["sigma1"], 1e-11) and _close(f2, ref["sigma2"], 1e-11)


def test_split_left_and_right_are_transposes(g):
    no, nv = 4, 24
    inp = make_inputs(no, nv, seed=35)
    R1, R2 = make_trial_vectors(no, nv, 2, seed=4)
    L1, L2 = make_trial_vectors(no, nv, 2, seed=6)
    ctx = g.Context(inp)
    r1, r2 = ctx.jacobian(R1, R2, [0.3, 0.3], g.CC3_SPLIT_BF16)
    s1, s2 = ctx.left_jacobian(L1, L2, [0.3, 0.3], g.CC3_SPLIT_BF16)
    for n in range(2):
        for m in range(2):
            a = np.sum(L1[n] * r1[m]) + np.sum(L2[n] * r2[m])
            b = np.sum(s1[n] * R1[m]) + np.sum(s2[n] * R2[m])
            assert abs(a - b) <= 1e-9


def test_split_left_jacobian_batched_shape(g):
    """The batched-Jacobian shape (no=20, nv=200, 96- and 48-column N tiles,
    several K splits) on a triple subset against the matrix-product oracle."""
    from oracle import matrix_form as MF
    inp = config_inputs("cfg4_jacobian_no20_nv200")
    no, nv = inp.no, inp.nv
    L1, L2 = make_trial_vectors(no, nv, 3, seed=13)
    w = [0.25, 0.0, -0.1]
    tr = [t[:3] for t in unique_triples(no)]
    rng = np.random.default_rng(10)
    sel = [tr[i] for i in sorted(rng.choice(len(tr), size=2, replace=False))] + [(18, 18, 3)]
    ref = MF.left_jacobian(inp, L1, L2, w, triples=sel)
    ctx = g.Context(inp)
    ctx.set_triples(sel)
    s1, s2 = ctx.left_jacobian(L1, L2, w, g.CC3_SPLIT_BF16)
    assert split_close(s1, ref["sigma1"]), split_err(s1, ref["sigma1"])
    assert split_close(s2, ref["sigma2"]), split_err(s2, ref["sigma2"])


def test_split_left_jacobian_device_pointers_and_cvs_subset(g):
    """Device pointers and a core-valence-separation triple list on the split path,
    against the oracle restricted to the same triples."""
    import torch
    no, nv = 5, 24
    inp = make_inputs(no, nv, seed=44)
    L1, L2 = make_trial_vectors(no, nv, 2, seed=7)
    ctx = g.Context(inp, device=True)
    tri = ctx.set_cvs([0, 1])
    ref = oracle.left_jacobian(inp, L1, L2, [0.2, -0.05], triples=[t[:3] for t in tri])
    s1, s2 = ctx.left_jacobian(torch.from_numpy(L1).cuda(), torch.from_numpy(L2).cuda(),
                               [0.2, -0.05], g.CC3_SPLIT_BF16)
    torch.cuda.synchronize()
    assert split_close(s1.cpu().numpy(), ref["sigma1"]), split_err(s1.cpu().numpy(), ref["sigma1"])
    assert split_close(s2.cpu().numpy(), ref["sigma2"]), split_err(s2.cpu().numpy(), ref["sigma2"])
