"""Denominator checks of the boundary: the host-only gap between a frequency
and the triples denominators eps^{abc}_{ijk} = e_a + e_b + e_c - e_i - e_j - e_k
(the R3 denominator (w - eps) of the Jacobian, eq. "jcc3"; at w = 0 the tau
denominator of Algorithm 1), checked against brute force over every (a, b, c)
and (i, j, k); the Jacobian's rejection of a frequency on a denominator (GPU)."""
import itertools
import os
import re

import numpy as np
import pytest

from cc3_inputs import make_inputs, make_trial_vectors, unique_triples

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def brute_gap(eo, ev, w, triples):
    abc = np.add.outer(np.add.outer(ev, ev), ev).ravel()
    return min(np.abs(w - (abc - (eo[i] + eo[j] + eo[k]))).min() for i, j, k in triples)


@pytest.mark.parametrize("no,nv,seed", [(3, 5, 0), (4, 7, 1), (5, 4, 2)])
def test_gap_matches_brute_force(no, nv, seed):
    import paper_2007_01088_gb300 as g
    rng = np.random.default_rng(seed)
    eo = np.sort(rng.uniform(-1.5, -0.3, no))
    ev = rng.uniform(0.1, 3.0, nv)  # unsorted on purpose
    full = [t[:3] for t in unique_triples(no)]
    sub = full[::2]
    # frequencies below, inside and above the denominators' range, and one a
    # tenth of a micro-hartree from a chosen denominator
    e0 = ev[1] + ev[2] + ev[nv - 1] - (eo[no - 1] + eo[0] + eo[0])
    for w in [0.0, 0.25, 2.0, 7.5, 20.0, -1.0, e0 + 1e-7]:
        for tri in (None, sub):
            ref = brute_gap(eo, ev, w, full if tri is None else sub)
            got = g.cc3_denominator_gap(no, nv, eo, ev, w, tri)
            assert abs(got - ref) <= 1e-14 * max(1.0, abs(w) + 10.0), (w, got, ref)
    assert g.cc3_denominator_gap(no, nv, eo, ev, e0 + 1e-7) < g.CC3_DENOM_MIN


def test_gap_of_ground_state_denominators_is_their_minimum():
    # w = 0 on the full loop: the smallest tau denominator, 3 min eps_v minus
    # the largest occupied sum of a triple that is not all equal
    import paper_2007_01088_gb300 as g
    inp = make_inputs(4, 9, seed=5)
    eo, ev = inp.eps_o, inp.eps_v
    top = max(eo[i] + eo[j] + eo[k] for i, j, k, _ in unique_triples(4))
    assert g.cc3_denominator_gap(4, 9, eo, ev, 0.0) == pytest.approx(3 * ev.min() - top,
                                                                   rel=1e-14)


def test_gap_empty_loop_and_argument_errors():
    import paper_2007_01088_gb300 as g
    eo, ev = np.array([-0.5]), np.array([0.3, 0.7])
    assert g.cc3_denominator_gap(1, 2, eo, ev, 0.0) == 1e300  # no = 1: no triple
    with pytest.raises(g.CC3Error) as e:
        g.cc3_denominator_gap(3, 2, np.array([-0.5, -0.4, -0.3]), ev, 0.0, [(0, 1, 0)])
    assert e.value.status == g.CC3_ERR_ARG  # triple not in i >= j >= k order
    with pytest.raises(g.CC3Error):
        g.cc3_denominator_gap(1, 2, eo, ev, float("nan"))
    with pytest.raises(g.CC3Error):
        g.cc3_denominator_gap(0, 2, eo, ev, 0.0)


def test_header_and_binding_share_the_threshold():
    import paper_2007_01088_gb300 as g
    txt = open(os.path.join(ROOT, "include", "cc3.h")).read()
    m = re.search(r"#define\s+CC3_DENOM_MIN\s+([0-9.eE+-]+)", txt)
    assert m and float(m.group(1)) == g.CC3_DENOM_MIN


@pytest.mark.gpu
def test_jacobian_rejects_frequency_on_a_denominator():
    import paper_2007_01088_gb300 as g
    no, nv = 3, 10
    inp = make_inputs(no, nv, seed=8)
    R1, R2 = make_trial_vectors(no, nv, 2, seed=2)
    eo, ev = inp.eps_o, inp.eps_v
    w_bad = ev[0] + ev[3] + ev[5] - (eo[2] + eo[1] + eo[0]) + 2e-7
    ctx = g.Context(inp)
    with pytest.raises(g.CC3Error) as e:
        ctx.jacobian(R1, R2, [0.25, w_bad], g.CC3_FP64)
    assert e.value.status == g.CC3_ERR_DENOM
    with pytest.raises(g.CC3Error) as e:
        ctx.jacobian(R1, R2, [w_bad, 0.0], g.CC3_SPLIT_BF16)
    assert e.value.status == g.CC3_ERR_DENOM
    # the context stays usable; a frequency clear of the denominators passes
    r1, _ = ctx.jacobian(R1, R2, [0.25, 0.0], g.CC3_FP64)
    assert np.isfinite(r1).all()
