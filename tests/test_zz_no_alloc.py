"""The no-allocation entry point (for callers that cannot call cudaMalloc,
such as code embedded in an application that owns the GPU memory pool) gives
the same residual as the context-based FP64 entry point.  Collected last."""
import numpy as np
import pytest

from cc3_inputs import make_inputs

pytestmark = pytest.mark.gpu

NAMES = ["eps_o", "eps_v", "t2", "g_vvvo", "g_ooov", "g_ovov", "F_ov"]


def _device(inp):
    import torch
    return {n: torch.from_numpy(np.ascontiguousarray(getattr(inp, n))).cuda() for n in NAMES}


def _call(g, no, nv, d):
    import torch
    o1 = torch.full((no, nv), float("nan"), dtype=torch.float64, device="cuda")
    o2 = torch.full((no, no, nv, nv), float("nan"), dtype=torch.float64, device="cuda")
    e = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    g.cc3_omega_triples_noalloc(no, nv, *[d[n] for n in NAMES], o1, o2, e)
    torch.cuda.synchronize()
    return o1.cpu().numpy(), o2.cpu().numpy(), e.cpu().numpy()


# (12, 64) is the documented size limit: its data and the contraction tables of
# all 352 triples must fit the 16 MiB array
@pytest.mark.parametrize("no,nv", [(5, 30), (4, 33), (12, 64)])
def test_noalloc_matches_context_path(no, nv):
    import paper_2007_01088_gb300 as g
    inp = make_inputs(no, nv, seed=3 * no + nv)
    ctx = g.Context(inp)
    ref1, ref2, refe = ctx.omega(g.CC3_FP64)
    ctx.close()
    d = _device(inp)
    for _ in range(2):  # two calls in a row share the scratch array
        o1, o2, e = _call(g, no, nv, d)
        assert np.abs(o1 - ref1).max() <= 1e-12 * np.abs(ref1).max()
        assert np.abs(o2 - ref2).max() <= 1e-12 * np.abs(ref2).max()
        assert abs(e[0] - refe[0]) <= 1e-12 * abs(refe[0])


def test_noalloc_single_occupied_orbital_gives_zero():
    # no = 1: every triple is i = j = k, the loop is empty; the outputs are
    # exact zeros even though an earlier call left other values in the array
    import paper_2007_01088_gb300 as g
    _call(g, 4, 20, _device(make_inputs(4, 20, seed=2)))
    o1, o2, e = _call(g, 1, 12, _device(make_inputs(1, 12, seed=1)))
    assert not o1.any() and not o2.any() and e[0] == 0.0


def test_noalloc_rejects_oversized_problem():
    import torch
    import paper_2007_01088_gb300 as g
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(g.CC3Error) as ex:
        g.cc3_omega_triples_noalloc(13, 10, z, z, z, z, z, z, z, None, None, None)
    assert ex.value.status == g.CC3_ERR_ARG


def test_noalloc_rejects_non_positive_denominators():
    # a virtual energy below the highest occupied one: some eps^{abc}_{ijk} <= 0
    import paper_2007_01088_gb300 as g
    inp = make_inputs(3, 10, seed=4)
    inp.eps_v = inp.eps_v.copy()
    inp.eps_v[0] = inp.eps_o.max() - 0.1
    with pytest.raises(g.CC3Error) as ex:
        _call(g, 3, 10, _device(inp))
    assert ex.value.status == g.CC3_ERR_DENOM
