"""General (T1-transformed) integrals through cc3_ctx_create_general: the five
blocks of Algorithm 1 given separately, without the 8-fold symmetry the
T1 = 0 inputs have (paper, "Implementation": the integrals are T1
transformed).  The library's residual on both precision paths against the
oracle's general five-block form on the same blocks."""
import numpy as np
import pytest

import oracle
from cc3_inputs import make_inputs, make_trial_vectors
from split_tol import energy_close, split_close, split_err


def _t1_blocks(no, nv, seed, scale=0.1):
    inp = make_inputs(no, nv, seed=seed)
    t1 = np.random.default_rng(seed + 1).normal(0.0, scale, size=(no, nv))
    return inp, oracle.t1_transform(inp, t1)


def test_general_create_rejects_missing_blocks_on_the_host():
    import ctypes
    import paper_2007_01088_gb300 as g
    ctx = ctypes.c_void_p()
    z = np.zeros(4)
    p = z.ctypes.data_as(ctypes.c_void_p)
    # g_oovo missing: rejected before any device work
    assert g.lib.cc3_ctx_create_general(ctypes.byref(ctx), 2, 2, p, p, p, p, None, p, p, p, p,
                                        0, None) == g.CC3_ERR_ARG
    assert g.lib.cc3_ctx_create_general(ctypes.byref(ctx), 0, 2, p, p, p, p, p, p, p, p, p,
                                        0, None) == g.CC3_ERR_ARG


def test_t1_transformed_blocks_are_not_symmetric():
    _, b = _t1_blocks(3, 8, 1)
    assert np.abs(b["vvvo"] - np.transpose(b["vvov"], (1, 0, 3, 2))).max() > 1e-4
    assert np.abs(b["oovo"] - np.transpose(b["ooov"], (0, 1, 3, 2))).max() > 1e-5


@pytest.mark.gpu
@pytest.mark.parametrize("no,nv", [(5, 30), (4, 70), (2, 9), (3, 136)])
def test_general_residual_matches_oracle(no, nv):
    import paper_2007_01088_gb300 as g
    from oracle import matrix_form as MF
    inp, b = _t1_blocks(no, nv, seed=no * nv)
    ref = MF.omega(no, nv, inp.eps_o, inp.eps_v, inp.t2, b)
    ctx = g.Context(inp, blocks=b)
    o1, o2, e = ctx.omega(g.CC3_FP64)
    s = max(np.abs(ref["omega2"]).max(), 1e-300)
    assert np.abs(o2 - ref["omega2"]).max() <= 1e-12 * s
    assert np.abs(o1 - ref["omega1"]).max() <= 1e-12 * np.abs(ref["omega1"]).max()
    assert abs(e[0] - ref["E_T"]) <= 1e-12 * abs(ref["E_T"])
    o1, o2, e = ctx.omega(g.CC3_SPLIT_BF16)
    assert split_close(o1, ref["omega1"]), split_err(o1, ref["omega1"])
    assert split_close(o2, ref["omega2"]), split_err(o2, ref["omega2"])
    assert energy_close(e[0], ref["E_T"]), (e[0], ref["E_T"])


@pytest.mark.gpu
def test_general_api_on_symmetric_blocks_equals_symmetric_api():
    import paper_2007_01088_gb300 as g
    inp = make_inputs(4, 33, seed=2)
    b = oracle.symmetric_blocks(inp)
    a = g.Context(inp).omega(g.CC3_FP64)
    c = g.Context(inp, blocks=b).omega(g.CC3_FP64)
    for x, y in zip(a, c):
        assert np.abs(x - y).max() <= 1e-13 * np.abs(x).max()


@pytest.mark.gpu
def test_general_context_triple_subset_and_jacobian_refusal():
    import paper_2007_01088_gb300 as g
    inp, b = _t1_blocks(5, 24, seed=7)
    sel = [(4, 2, 1), (3, 3, 0), (2, 1, 1)]
    ref = oracle.omega(5, 24, inp.eps_o, inp.eps_v, inp.t2, b, triples=sel)
    ctx = g.Context(inp, blocks=b)
    ctx.set_triples(sel)
    o1, o2, e = ctx.omega(g.CC3_SPLIT_BF16)
    assert split_close(o2, ref["omega2"]) and energy_close(e[0], ref["E_T"])
    R1, R2 = make_trial_vectors(5, 24, 1)
    with pytest.raises(g.CC3Error) as err:
        ctx.jacobian(R1, R2, [0.0], g.CC3_FP64)
    assert err.value.status == g.CC3_ERR_UNSUPPORTED
