"""Split-precision (BF16 slice) tensor-core path against FP64 references.
Calls go through the C ABI.  Tolerances are the split path's targets, 1e-9
absolute on Omega and 1e-8 Eh on the triples energy, each also held to 1e-10
of the reference's largest magnitude (split_tol)."""
import numpy as np
import pytest

import oracle
from cc3_inputs import make_inputs, unique_triples
from split_tol import energy_close, split_close, split_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2007_01088_gb300 as g
    return g


@pytest.mark.parametrize("M,N,K", [(128, 160, 64), (200, 96, 700), (64, 32, 16),
                                   (300, 130, 1040), (17, 5, 33)])
def test_engine_gemm_matches_fp64(g, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(size=(M, K)) * np.exp(rng.normal(size=(M, 1)))
    B = rng.normal(size=(N, K))
    ref = A @ B.T
    scale = np.abs(A).max() * np.abs(B).max() * K
    C = g.cc3_debug_split_gemm(A, B, 6)
    assert np.abs(C - ref).max() <= 1e-13 * scale
    C3 = g.cc3_debug_split_gemm(A, B, 3)
    assert np.abs(C3 - ref).max() <= 1e-6 * scale
    C7 = g.cc3_debug_split_gemm(A, B, 7)
    assert np.abs(C7 - ref).max() <= 1e-15 * scale


def test_engine_gemm_exact_integers(g):
    # small integers are represented exactly by the first slice: exact result
    rng = np.random.default_rng(1)
    A = rng.integers(-100, 100, size=(130, 600)).astype(np.float64)
    B = rng.integers(-100, 100, size=(64, 600)).astype(np.float64)
    assert np.array_equal(g.cc3_debug_split_gemm(A, B, 4), A @ B.T)


# (3, 160) and (4, 136): nv >= 128 with a remainder, the case where the vvov
# contraction stacks permutations along M (tiles holding two permutations)
@pytest.mark.parametrize("no,nv", [(5, 30), (4, 70), (3, 17), (6, 33), (3, 160), (4, 136)])
def test_omega_split_matches_oracle(g, no, nv):
    inp = make_inputs(no, nv, seed=no * nv)
    ref = oracle.omega_inputs(inp)
    ctx = g.Context(inp)
    o1, o2, e = ctx.omega(g.CC3_SPLIT_BF16)
    assert split_close(o1, ref["omega1"]), split_err(o1, ref["omega1"])
    assert split_close(o2, ref["omega2"]), split_err(o2, ref["omega2"])
    assert energy_close(e[0], ref["E_T"]), (e[0], ref["E_T"])
    c = ctx.counters()
    assert c["slices"] == 6 and c["executed_flop"] > c["nominal_flop"]


def test_omega_split_wide_dynamic_range(g):
    # each tensor is sliced with one power-of-two scale, so its small elements
    # keep fewer bits: t2 pair blocks and an occupied slab of the vvvo integrals
    # scaled down by 1e-3 to 1e-6 make the operands span up to six more orders of
    # magnitude, and the result must still meet the absolute and relative gates
    import dataclasses
    base = make_inputs(4, 40, seed=77)
    t2 = base.t2.copy()
    t2[1, 1] *= 1.0e-6
    t2[2, 0] *= 1.0e-3
    t2[0, 2] *= 1.0e-3  # keeps t2[i][j][a][b] = t2[j][i][b][a]
    vvvo = base.g_vvvo.copy()
    vvvo[:, :, :, 2] *= 1.0e-4
    inp = dataclasses.replace(base, t2=t2, g_vvvo=vvvo)
    ref = oracle.omega_inputs(inp)
    o1, o2, e = g.Context(inp).omega(g.CC3_SPLIT_BF16)
    assert split_close(o1, ref["omega1"]), split_err(o1, ref["omega1"])
    assert split_close(o2, ref["omega2"]), split_err(o2, ref["omega2"])
    assert energy_close(e[0], ref["E_T"]), (e[0], ref["E_T"])


def test_autotune_keeps_parity_and_is_shared(g):
    inp = make_inputs(6, 40, seed=12)
    ref = oracle.omega_inputs(inp)
    ctx = g.Context(inp)
    ks, nt = ctx.autotune()
    assert ks in (200, 400, 800) and nt % 16 == 0 and 16 <= nt <= 96
    o1, o2, e = ctx.omega(g.CC3_SPLIT_BF16)
    assert split_close(o1, ref["omega1"]), split_err(o1, ref["omega1"])
    assert split_close(o2, ref["omega2"]), split_err(o2, ref["omega2"])
    assert energy_close(e[0], ref["E_T"]), (e[0], ref["E_T"])
    ctx2 = g.Context(inp)  # a later context of the same size starts tuned
    assert ctx2.tuning() == (ks, nt)


def test_split_edge_cases_small_no(g):
    # no = 1: the loop is empty (i = j = k only); no = 2: only weight-3 triples
    for no, nv in [(1, 12), (2, 9)]:
        inp = make_inputs(no, nv, seed=5 + no)
        ref = oracle.omega_inputs(inp)
        ctx = g.Context(inp)
        o1, o2, e = ctx.omega(g.CC3_SPLIT_BF16)
        if no == 1:  # empty loop: exact zeros
            assert not o1.any() and not o2.any() and e[0] == 0.0
            continue
        assert split_close(o1, ref["omega1"]), split_err(o1, ref["omega1"])
        assert split_close(o2, ref["omega2"]), split_err(o2, ref["omega2"])
        assert energy_close(e[0], ref["E_T"]), (e[0], ref["E_T"])


def test_split_proline_sized_triple_subset(g):
    # the L-proline-sized problem (22 active occupied, nv = 250, naux = 700,
    # near-degenerate virtual cluster): a seeded sample of triples against the
    # oracle restricted to the same triples
    inp = make_inputs(22, 250, seed=0, naux=700, nfrozen=9, n_degenerate=10)
    tr = unique_triples(22)
    rng = np.random.default_rng(3)
    sel = [tr[i][:3] for i in sorted(rng.choice(len(tr), size=3, replace=False))]
    sel.append((21, 21, 20))  # a weight-3 triple at the top of the range
    ref = oracle.omega_inputs(inp, triples=sel)
    ctx = g.Context(inp)
    ctx.set_triples(sel)
    o1, o2, e = ctx.omega(g.CC3_SPLIT_BF16)
    assert split_close(o1, ref["omega1"]), split_err(o1, ref["omega1"])
    assert split_close(o2, ref["omega2"]), split_err(o2, ref["omega2"])
    assert energy_close(e[0], ref["E_T"]), (e[0], ref["E_T"])


def test_graph_replay_matches_direct_launches(g):
    # untraced calls on a non-default stream: the second call captures the
    # launch sequence as a CUDA graph, later calls replay it
    import torch
    inp = make_inputs(5, 40, seed=21)
    ref = oracle.omega_inputs(inp)
    st = torch.cuda.Stream()
    ctx = g.Context(inp, stream=st)
    outs = [ctx.omega(g.CC3_SPLIT_BF16) for _ in range(4)]
    for o1, o2, e in outs:
        assert split_close(o1, ref["omega1"]), split_err(o1, ref["omega1"])
        assert split_close(o2, ref["omega2"]), split_err(o2, ref["omega2"])
        assert energy_close(e[0], ref["E_T"]), (e[0], ref["E_T"])
        assert np.abs(o2 - outs[0][1]).max() <= 1e-12 * np.abs(outs[0][1]).max()
    assert ctx.counters()["launches"] > 0
