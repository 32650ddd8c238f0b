"""FP64 path of the library against the FP64 oracle (tolerance 1e-12 in the
max norm relative to max|Omega_oracle|, the bound the hot path's FP64 target
states).  Calls go through the C ABI."""
import numpy as np
import pytest

import oracle
from cc3_inputs import make_inputs, unique_triples
from split_tol import energy_close, split_close

pytestmark = pytest.mark.gpu
TOL = 1e-12


def rel(a, b):
    return np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def g():
    import paper_2007_01088_gb300 as g
    return g


@pytest.mark.parametrize("no,nv", [(5, 30), (4, 70), (3, 65), (2, 9), (6, 17)])
def test_omega_fp64_matches_oracle(g, no, nv):
    inp = make_inputs(no, nv, seed=no + nv)
    ref = oracle.omega_inputs(inp)
    ctx = g.Context(inp)
    o1, o2, e = ctx.omega(g.CC3_FP64)
    assert rel(o1, ref["omega1"]) < TOL
    assert rel(o2, ref["omega2"]) < TOL
    assert abs(e[0] - ref["E_T"]) <= TOL * abs(ref["E_T"])
    c = ctx.counters()
    assert c["nominal_flop"] == 4 * nv ** 4 * (no ** 3 - no)
    assert c["launches"] > 0


def test_no1_is_zero(g):
    inp = make_inputs(1, 12, 0)
    o1, o2, e = g.Context(inp).omega(g.CC3_FP64)
    assert np.all(o1 == 0) and np.all(o2 == 0) and e[0] == 0


def test_device_pointer_mode(g):
    import torch
    inp = make_inputs(4, 33, 1)
    ref = oracle.omega_inputs(inp)
    ctx = g.Context(inp, device=True)
    o1, o2, e = ctx.omega(g.CC3_FP64)
    torch.cuda.synchronize()
    assert o2.is_cuda
    assert rel(o2.cpu().numpy(), ref["omega2"]) < TOL
    assert abs(e.item() - ref["E_T"]) <= TOL * abs(ref["E_T"])


def test_triple_subset_at_full_size(g):
    # no = 16, nv = 160 (the headline workload's shape); a seeded sample of
    # triples on both sides, including both permutation classes
    inp = make_inputs(16, 160, 0)
    tr = [t[:3] for t in unique_triples(16)]
    rng = np.random.default_rng(7)
    sel = [tr[x] for x in sorted(rng.choice(len(tr), 3, replace=False))] + [(15, 15, 3)]
    ref = oracle.omega_inputs(inp, triples=sel)
    ctx = g.Context(inp)
    ctx.set_triples(sel)
    o1, o2, e = ctx.omega(g.CC3_FP64)
    assert rel(o1, ref["omega1"]) < TOL
    assert rel(o2, ref["omega2"]) < TOL
    assert abs(e[0] - ref["E_T"]) <= TOL * abs(ref["E_T"])


def test_subsets_add_up(g):
    inp = make_inputs(6, 40, 2)
    tr = [t[:3] for t in unique_triples(6)]
    ctx = g.Context(inp)
    full = [x.copy() for x in ctx.omega(g.CC3_FP64)]
    ctx.set_triples(tr[::2])
    a = [x.copy() for x in ctx.omega(g.CC3_FP64)]
    ctx.set_triples(tr[1::2])
    b = [x.copy() for x in ctx.omega(g.CC3_FP64)]
    assert rel(a[1] + b[1], full[1]) < 1e-13
    assert abs(a[2][0] + b[2][0] - full[2][0]) < 1e-13 * abs(full[2][0])


@pytest.mark.parametrize("split", [False, True])
def test_deterministic_mode_is_bitwise_reproducible(g, split):
    # CC3_DETERMINISTIC: the cross-triple sums accumulate in 128-bit fixed
    # point, so repeated evaluations agree bit for bit (FP64 atomics would
    # agree only to rounding)
    inp = make_inputs(6, 40, seed=31)
    ref = oracle.omega_inputs(inp)
    prec = g.CC3_SPLIT_BF16 if split else g.CC3_FP64
    ctx = g.Context(inp, flags=g.CC3_DETERMINISTIC)
    runs = [ctx.omega(prec) for _ in range(3)]
    ctx2 = g.Context(inp, flags=g.CC3_DETERMINISTIC)
    runs.append(ctx2.omega(prec))
    for o1, o2, e in runs[1:]:
        assert np.array_equal(o1, runs[0][0]) and np.array_equal(o2, runs[0][1])
        assert e[0] == runs[0][2][0]
    o1, o2, e = runs[0]
    if split:
        assert split_close(o2, ref["omega2"]) and energy_close(e[0], ref["E_T"])
    else:
        assert np.abs(o2 - ref["omega2"]).max() <= 1e-12 * np.abs(ref["omega2"]).max()
        assert abs(e[0] - ref["E_T"]) <= 1e-12 * abs(ref["E_T"])
    from cc3_inputs import make_trial_vectors
    R1, R2 = make_trial_vectors(6, 40, 1)
    with pytest.raises(g.CC3Error) as err:
        ctx.jacobian(R1, R2, [0.0], prec)
    assert err.value.status == g.CC3_ERR_UNSUPPORTED
