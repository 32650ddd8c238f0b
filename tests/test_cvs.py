"""Core-valence separation task filter (paper, Introduction and Applications:
the triple loop skips the occupied triples that contain no core orbital of
interest).  The filter itself runs on the host (no GPU); the oracle pins that
restricting the tasks is an exact partition of the triples sum; the GPU test
compares the library's filtered Jacobian with the oracle on the same tasks."""
import numpy as np
import pytest

import oracle
from cc3_inputs import make_inputs, make_trial_vectors, unique_triples
from split_tol import split_close, split_err


def _enumerate(no, core):
    cs = set(core)
    return [(i, j, k) for (i, j, k, _) in unique_triples(no) if cs & {i, j, k}]


@pytest.mark.parametrize("no,core", [(1, [0]), (2, [0]), (4, [0]), (5, [1, 3]),
                                     (6, []), (7, [0, 1, 2, 3, 4, 5, 6])])
def test_cvs_triples_match_definition(no, core):
    import paper_2007_01088_gb300 as g
    tr = g.cc3_cvs_triples(no, core)
    assert [tuple(int(x) for x in t) for t in tr] == _enumerate(no, core)


@pytest.mark.parametrize("no,ncore", [(3, 1), (8, 1), (8, 2), (12, 3)])
def test_cvs_task_weight_is_the_core_containing_ordered_triples(no, ncore):
    # distinct permutations of the kept triples = ordered triples with at least
    # one core index, minus the core diagonal i = j = k; for one core orbital
    # 3 no^2 - 3 no, the 8 nv^4 no^2 scaling of the paper's CVS Jacobian
    import paper_2007_01088_gb300 as g
    core = list(range(ncore))
    w = dict(((i, j, k), wt) for (i, j, k, wt) in unique_triples(no))
    kept = [tuple(int(x) for x in t) for t in g.cc3_cvs_triples(no, core)]
    total = sum(w[t] for t in kept)
    assert total == no ** 3 - (no - ncore) ** 3 - ncore
    if ncore == 1:
        assert total == 3 * no * no - 3 * no


def test_cvs_triples_reject_bad_core():
    import paper_2007_01088_gb300 as g
    for no, core in [(4, [4]), (4, [-1]), (4, [1, 1]), (2, [0, 1, 0])]:
        with pytest.raises(g.CC3Error):
            g.cc3_cvs_triples(no, core)
    assert g.lib.cc3_cvs_triples(3, 4, None, 0, None) == g.CC3_ERR_ARG
    assert g.lib.cc3_cvs_triples(-1, 0, None, 0, None) == g.CC3_ERR_ARG


def test_task_partition_is_exact_in_the_oracle():
    # the Jacobian (and the residual) over all triples is the sum over the
    # core-containing triples and over the rest
    no, nv = 4, 6
    inp = make_inputs(no, nv, seed=2)
    R1, R2 = make_trial_vectors(no, nv, 2, seed=2)
    w = [0.25, 0.0]
    core = [0]
    cvs = _enumerate(no, core)
    rest = [t[:3] for t in unique_triples(no) if tuple(t[:3]) not in set(cvs)]
    full = oracle.jacobian(inp, R1, R2, w)
    a = oracle.jacobian(inp, R1, R2, w, triples=cvs)
    b = oracle.jacobian(inp, R1, R2, w, triples=rest)
    for key in ("rho1", "rho2"):
        scale = np.abs(full[key]).max()
        assert np.abs(a[key] + b[key] - full[key]).max() <= 1e-13 * scale
        assert np.abs(a[key]).max() > 1e-3 * scale  # the filtered part is not empty
    fo = oracle.omega_inputs(inp)
    ao = oracle.omega_inputs(inp, triples=cvs)
    bo = oracle.omega_inputs(inp, triples=rest)
    assert abs(ao["E_T"] + bo["E_T"] - fo["E_T"]) <= 1e-13 * abs(fo["E_T"])


# (4, 136): nv >= 128, where the split path's vvov tiles stack two permutations
@pytest.mark.gpu
@pytest.mark.parametrize("prec_name", ["CC3_FP64", "CC3_SPLIT_BF16"])
@pytest.mark.parametrize("no,nv", [(5, 24), (4, 136)])
def test_cvs_jacobian_matches_oracle_on_the_same_tasks(prec_name, no, nv):
    import paper_2007_01088_gb300 as g
    from oracle import matrix_form as MF
    inp = make_inputs(no, nv, seed=4)
    R1, R2 = make_trial_vectors(no, nv, 2, seed=4)
    w = [0.25, 0.0]
    ctx = g.Context(inp)
    tr = ctx.set_cvs([0])
    ref = MF.jacobian(inp, R1, R2, w, triples=[tuple(int(x) for x in t) for t in tr])
    r1, r2 = ctx.jacobian(R1, R2, w, getattr(g, prec_name))
    ctx.close()
    if prec_name == "CC3_FP64":
        assert np.abs(r1 - ref["rho1"]).max() <= 1e-12 * np.abs(ref["rho1"]).max()
        assert np.abs(r2 - ref["rho2"]).max() <= 1e-12 * np.abs(ref["rho2"]).max()
    else:
        assert split_close(r1, ref["rho1"]), split_err(r1, ref["rho1"])
        assert split_close(r2, ref["rho2"]), split_err(r2, ref["rho2"])
