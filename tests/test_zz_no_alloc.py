"""The no-allocation entry point (for callers that cannot call cudaMalloc,
such as code embedded in an application that owns the GPU memory pool) gives
the same residual as the context-based FP64 entry point.  Collected last."""
import numpy as np
import pytest

from cc3_inputs import make_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("no,nv", [(5, 30), (4, 33)])
def test_noalloc_matches_context_path(no, nv):
    import torch
    import paper_2007_01088_gb300 as g
    inp = make_inputs(no, nv, seed=3 * no + nv)
    ctx = g.Context(inp)
    ref1, ref2, refe = ctx.omega(g.CC3_FP64)
    ctx.close()
    d = {n: torch.from_numpy(np.ascontiguousarray(getattr(inp, n))).cuda()
         for n in ["eps_o", "eps_v", "t2", "g_vvvo", "g_ooov", "g_ovov", "F_ov"]}
    for _ in range(2):  # two calls in a row share the scratch array
        o1 = torch.full((no, nv), float("nan"), dtype=torch.float64, device="cuda")
        o2 = torch.full((no, no, nv, nv), float("nan"), dtype=torch.float64, device="cuda")
        e = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        g.cc3_omega_triples_noalloc(no, nv, d["eps_o"], d["eps_v"], d["t2"], d["g_vvvo"],
                                    d["g_ooov"], d["g_ovov"], d["F_ov"], o1, o2, e)
        torch.cuda.synchronize()
        o1, o2, e = o1.cpu().numpy(), o2.cpu().numpy(), e.cpu().numpy()
        assert np.abs(o1 - ref1).max() <= 1e-12 * np.abs(ref1).max()
        assert np.abs(o2 - ref2).max() <= 1e-12 * np.abs(ref2).max()
        assert abs(e[0] - refe[0]) <= 1e-12 * abs(refe[0])


def test_noalloc_rejects_oversized_problem():
    import torch
    import paper_2007_01088_gb300 as g
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(g.CC3Error) as ex:
        g.cc3_omega_triples_noalloc(13, 10, z, z, z, z, z, z, z, None, None, None)
    assert ex.value.status == -1
