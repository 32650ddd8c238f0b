"""Right CC3 Jacobian transformation (triples part) through the C ABI against
the oracle (eq. "jcc3" with the Algorithm 2 intermediates on the GPU side, the
direct tau~3 . g^ contractions on the oracle side).

FP64 path: 1e-11 relative to the largest element of the reference, elementwise
(a few hundred FP64 roundings in the longest sums, well below that bound).
Split path: the residual's absolute target, 1e-9 (the trial vectors are
normalised, so rho has the residual's scale), and 1e-10 of the largest
reference element (split_tol).

The batched-Jacobian shape (no = 20, nv = 200, naux = 660, 8 trial vectors)
is checked on a seeded triple subset against the matrix-product form of the
oracle (oracle.matrix_form, pinned to the C oracle), whose C loops would take
minutes per triple there."""
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


@pytest.mark.parametrize("no,nv", [(3, 9), (4, 20), (5, 33), (3, 40)])
def test_jacobian_split_matches_oracle(g, no, nv):
    inp = make_inputs(no, nv, seed=300 + no * nv)
    R1, R2 = make_trial_vectors(no, nv, 3, seed=no * nv)
    w = [0.25, 0.0, -0.1]
    ref = oracle.jacobian(inp, R1, R2, w)
    ctx = g.Context(inp)
    r1, r2 = ctx.jacobian(R1, R2, w, g.CC3_SPLIT_BF16)
    assert split_close(r1, ref["rho1"]), split_err(r1, ref["rho1"])
    assert split_close(r2, ref["rho2"]), split_err(r2, ref["rho2"])
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
        assert split_close(x, y), split_err(x, y)


# the batched-Jacobian workload's shape: 8 trial vectors at several
# frequencies, nv = 200 (vvov tiles stacking two permutations, 96-column N
# tiles, the Cholesky term of the dressed vvvo block on the tensor cores), on
# a seeded subset of triples that includes a weight-3 triple
W8 = [0.25, 0.0, -0.1, 0.3, 0.25, 0.1, 0.0, 0.2]
CHECK = [0, 2, 7]  # vectors checked against the oracle; all 8 split vs FP64


def test_jacobian_batched_shape_both_paths(g):
    from oracle import matrix_form as MF
    inp = config_inputs("cfg4_jacobian_no20_nv200")
    no, nv = inp.no, inp.nv
    assert (no, nv, inp.naux) == (20, 200, 660)
    R1, R2 = make_trial_vectors(no, nv, 8, seed=1)
    tr = [t[:3] for t in unique_triples(no)]
    rng = np.random.default_rng(5)
    sel = [tr[i] for i in sorted(rng.choice(len(tr), size=3, replace=False))] + [(19, 19, 4)]
    ref = MF.jacobian(inp, R1[CHECK], R2[CHECK], [W8[n] for n in CHECK], triples=sel)
    ctx = g.Context(inp)
    ctx.set_triples(sel)
    f1, f2 = ctx.jacobian(R1, R2, W8, g.CC3_FP64)
    s1, s2 = ctx.jacobian(R1, R2, W8, g.CC3_SPLIT_BF16)
    for u, n in enumerate(CHECK):
        assert _close(f1[n], ref["rho1"][u], 1e-11)
        assert _close(f2[n], ref["rho2"][u], 1e-11)
        assert split_close(s1[n], ref["rho1"][u]), split_err(s1[n], ref["rho1"][u])
        assert split_close(s2[n], ref["rho2"][u]), split_err(s2[n], ref["rho2"][u])
    for n in range(8):
        assert split_close(s1[n], f1[n]), (n, split_err(s1[n], f1[n]))
        assert split_close(s2[n], f2[n]), (n, split_err(s2[n], f2[n]))


def test_split_jacobian_launches_per_batch_do_not_grow_with_vectors(g):
    # every phase of a batch of triples is one launch for all trial vectors:
    # the launches that grow with nvec are the per-vector set-up (dressing,
    # slicing, the Z~ . R1 terms), the same for any number of triples
    no, nv = 6, 20
    inp = make_inputs(no, nv, seed=61)
    tr = [t[:3] for t in unique_triples(no)]
    counts = {}
    for ntri in (4, len(tr)):
        for nvec in (1, 4):
            R1, R2 = make_trial_vectors(no, nv, nvec, seed=nvec)
            ctx = g.Context(inp)
            ctx.set_triples(tr[:ntri])
            ctx.jacobian(R1, R2, [0.2] * nvec, g.CC3_SPLIT_BF16)  # fills the Z~ cache
            ctx.jacobian(R1, R2, [0.2] * nvec, g.CC3_SPLIT_BF16)
            counts[(ntri, nvec)] = ctx.counters()["launches"]
            ctx.close()
    assert counts[(4, 4)] - counts[(4, 1)] == counts[(len(tr), 4)] - counts[(len(tr), 1)]
    assert counts[(len(tr), 1)] > counts[(4, 1)]
