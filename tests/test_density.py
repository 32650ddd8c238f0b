"""Algorithm 3: the triples contributions to the one-electron density of a
left state.

CPU part (pins of the oracle, nothing here touches the GPU):
- the restricted loops (occupied i >= j >= k, virtual a >= b >= c) equal the
  plain full-tensor sums;
- the vv and oo blocks at w = 0 are the derivatives of sum L.Omega with
  respect to a one-electron perturbation of the virtual-virtual or
  occupied-occupied Fock block inside the triples equations (complex step
  through a direct solve of the perturbed triples equations);
- the L2 part of the ov block is the derivative of sum L.Omega with respect
  to F_kc (Omega is linear in F_ov);
- tr Dvv + tr Doo = 0 (the two loops, different index restrictions);
- no = 1 and nv = 1 give zero; linearity in the left state; the FLOP count.

GPU part (marked gpu): the library's FP64 density through the C ABI against
the oracle, 1e-11 relative to the largest element of each block; the split
(BF16 slice) density with a left state normalised like the trial vectors,
within the split path's absolute and relative targets.
"""
import numpy as np
import pytest

import oracle
from oracle import definition as D
from cc3_inputs import make_inputs, make_trial_vectors
from split_tol import split_close, split_err


def _left(no, nv, seed):
    rng = np.random.default_rng(seed)
    L2 = rng.normal(size=(no, no, nv, nv))
    return rng.normal(size=(no, nv)), 0.5 * (L2 + np.transpose(L2, (1, 0, 3, 2)))


def _rel(x, ref):
    return np.abs(np.asarray(x) - ref).max() / max(np.abs(ref).max(), 1e-300)


def _density(inp, w, L1, L2):
    return oracle.density_inputs(inp, w, L1, L2)


def _pairing(inp, blocks, L1, L2, tau):
    """sum L1.Omega1 + sum L2.Omega2 for the residual built from tau."""
    om1, omt = D.contractions(D.contravariant(tau), blocks)
    return np.sum(L1 * om1) + np.sum(L2 * D.back_transform(omt))


@pytest.mark.parametrize("no,nv", [(2, 3), (3, 4), (4, 3), (3, 5)])
def test_restricted_loops_equal_full_sums(no, nv):
    inp = make_inputs(no, nv, seed=10 * no + nv)
    L1, L2 = _left(no, nv, seed=no * nv)
    b = oracle.symmetric_blocks(inp)
    for w in (0.0, 0.41):
        r = _density(inp, w, L1, L2)
        d = D.density_full(inp.eps_o, inp.eps_v, inp.t2, b, w, L1, L2)
        for k in ("Doo", "Dov", "Dvv"):
            assert _rel(r[k], d[k]) < 1e-13, k


def test_restricted_loops_general_blocks():
    """Non-symmetric (T1-transformed) blocks: the loops still equal the sums."""
    no, nv = 3, 4
    inp = make_inputs(no, nv, seed=5, naux=20)
    rng = np.random.default_rng(8)
    b = oracle.t1_transform(inp, 0.1 * rng.normal(size=(no, nv)))
    L1, L2 = _left(no, nv, seed=9)
    r = oracle.density(no, nv, inp.eps_o, inp.eps_v, inp.t2, b, 0.2, L1, L2)
    d = D.density_full(inp.eps_o, inp.eps_v, inp.t2, b, 0.2, L1, L2)
    for k in ("Doo", "Dov", "Dvv"):
        assert _rel(r[k], d[k]) < 1e-13, k


def _perturbed_tau(inp, blocks, block, p, q, h):
    """tau solving the triples equations with the one-electron operator
    F0 + h E_pq (F0 = the orbital energies): (eps + h K) tau = -W, with K the
    action of [E_pq, .] on the virtual (block 'vv') or occupied ('oo') indices
    of a triples tensor, solved directly for every fixed index set."""
    no, nv = inp.no, inp.nv
    W = D.W_full(inp.t2, blocks["vvvo"], blocks["oovo"])
    eps = D.denominators(inp.eps_o, inp.eps_v)
    tau = np.zeros(W.shape, dtype=complex)
    if block == "vv":
        f = np.zeros((nv, nv))
        f[p, q] = 1.0
        I = np.eye(nv)
        K = np.kron(np.kron(f, I), I) + np.kron(np.kron(I, f), I) + np.kron(np.kron(I, I), f)
        for i in range(no):
            for j in range(no):
                for k in range(no):
                    A = np.diag(eps[i, j, k].reshape(-1)) + h * K
                    tau[i, j, k] = np.linalg.solve(A, -W[i, j, k].reshape(-1)).reshape(nv, nv, nv)
    else:
        # [E_pq, E_ai] = -delta_pi E_aq: amplitude at occupied q receives -h tau(at p)
        g = np.zeros((no, no))
        g[q, p] = -1.0
        I = np.eye(no)
        K = np.kron(np.kron(g, I), I) + np.kron(np.kron(I, g), I) + np.kron(np.kron(I, I), g)
        Wt = np.moveaxis(W, (3, 4, 5), (0, 1, 2))
        et = np.moveaxis(eps, (3, 4, 5), (0, 1, 2))
        tt = np.zeros(Wt.shape, dtype=complex)
        for a in range(nv):
            for bb in range(nv):
                for c in range(nv):
                    A = np.diag(et[a, bb, c].reshape(-1)) + h * K
                    tt[a, bb, c] = np.linalg.solve(A, -Wt[a, bb, c].reshape(-1)).reshape(no, no, no)
        tau = np.moveaxis(tt, (0, 1, 2), (3, 4, 5))
    return tau


@pytest.mark.parametrize("no,nv", [(2, 3), (3, 3)])
def test_vv_and_oo_blocks_are_fock_derivatives(no, nv):
    inp = make_inputs(no, nv, seed=77 + no)
    L1, L2 = _left(no, nv, seed=3)
    b = oracle.symmetric_blocks(inp)
    r = _density(inp, 0.0, L1, L2)
    h = 1e-20
    dvv = np.zeros((nv, nv))
    for c in range(nv):
        for d in range(nv):
            tau = _perturbed_tau(inp, b, "vv", c, d, 1j * h)
            dvv[c, d] = np.imag(_pairing(inp, b, L1, L2, tau)) / h
    doo = np.zeros((no, no))
    for l in range(no):
        for k in range(no):
            tau = _perturbed_tau(inp, b, "oo", l, k, 1j * h)
            doo[l, k] = np.imag(_pairing(inp, b, L1, L2, tau)) / h
    assert _rel(r["Dvv"], dvv) < 1e-11
    assert _rel(r["Doo"], doo) < 1e-11


def test_ov_block_l2_part_is_the_F_derivative():
    no, nv = 3, 4
    inp = make_inputs(no, nv, seed=21)
    L1, L2 = _left(no, nv, seed=22)
    b = oracle.symmetric_blocks(inp)
    r = _density(inp, 0.3, L1, L2)
    d = D.density_full(inp.eps_o, inp.eps_v, inp.t2, b, 0.3, L1, L2)
    y_part = -np.einsum("clik,kicd->ld", d["Y"], inp.t2)

    def pairing(F):
        bb = dict(b)
        bb["F_ov"] = F
        o = oracle.omega(no, nv, inp.eps_o, inp.eps_v, inp.t2, bb)
        return np.sum(L1 * o["omega1"]) + np.sum(L2 * o["omega2"])

    base = pairing(np.zeros((no, nv)))
    dF = np.zeros((no, nv))
    for k in range(no):
        for c in range(nv):
            F = np.zeros((no, nv))
            F[k, c] = 1.0
            dF[k, c] = pairing(F) - base
    assert _rel(r["Dov"] - y_part, dF) < 1e-11
    assert np.abs(y_part).max() > 1e-3 * np.abs(dF).max()  # both parts present


@pytest.mark.parametrize("no,nv", [(4, 7), (5, 6)])
def test_trace_of_the_two_loops_cancels(no, nv):
    inp = make_inputs(no, nv, seed=no + nv)
    L1, L2 = _left(no, nv, seed=1)
    r = _density(inp, 0.15, L1, L2)
    tv, to = np.trace(r["Dvv"]), np.trace(r["Doo"])
    assert abs(tv) > 0 and abs(tv + to) <= 1e-12 * abs(tv)


def test_degenerate_sizes_give_zero():
    """no = 1: only i = j = k, where L~3 and tau~3 vanish; nv = 1: the same for
    a = b = c.  What is left is the rounding of sums that cancel exactly (the
    six terms of P in different orders): ~1e-38 here, against densities of
    ~1e-5 at the sizes above."""
    for no, nv in [(1, 5), (4, 1)]:
        inp = make_inputs(no, nv, seed=2)
        L1, L2 = _left(no, nv, seed=2)
        r = _density(inp, 0.1, L1, L2)
        for k in ("Doo", "Dov", "Dvv"):
            assert np.abs(r[k]).max() < 1e-30, (no, nv, k)


@pytest.mark.parametrize("no,nv", [(4, 5), (3, 6)])
def test_doo_by_occupied_pairs_equals_the_full_sum(no, nv):
    """The split path's D_oo reading: D_oo[l][k] = -1/2 sum_{ij} <L3~_{ijk}, tau_{ijl}>
    over (a,b,c), and because L3~ and tau are unchanged by a simultaneous swap of
    (i,a) with (j,b), the pair (j,i) repeats the sum of (i,j): the pairs i > j with
    weight 2 and i = j with weight 1 give the same block.  L3~ vanishes at
    i = j = k, which the split path uses as zero rows."""
    inp = make_inputs(no, nv, seed=no * nv)
    L1, L2 = _left(no, nv, seed=3)
    full = D.density_full(inp.eps_o, inp.eps_v, inp.t2, oracle.symmetric_blocks(inp), 0.2,
                          L1, L2)
    Lc, tau = D.contravariant(full["L3"]), full["tau"]
    pairs = np.zeros((no, no))
    for i in range(no):
        for j in range(i + 1):
            w = 1.0 if i == j else 2.0
            pairs += -0.5 * w * np.einsum("kabc,labc->lk", Lc[i, j], tau[i, j])
    assert _rel(pairs, full["Doo"]) < 1e-13
    swapped = np.einsum("ijkabc->jikbac", Lc)
    assert _rel(swapped, Lc) < 1e-13
    for i in range(no):
        assert np.abs(Lc[i, i, i]).max() <= 1e-13 * np.abs(Lc).max()


def test_symmetries_the_split_outer_products_read():
    """The split path forms the outer products of L3 (left transformation and
    densities) reading (o1 y|o2 z) as (o2 z|o1 y) and Lt2[o0][o1][x][y] as
    Lt2[o1][o0][y][x]: the symmetric integrals have the first symmetry, and the
    back-transform makes Lt2 pair symmetric for any L2."""
    inp = make_inputs(4, 9, seed=8)
    ov = inp.g_ovov
    assert np.abs(ov - np.transpose(ov, (2, 3, 0, 1))).max() <= 1e-15 * np.abs(ov).max()
    L2 = np.random.default_rng(9).normal(size=(4, 4, 9, 9))  # not pair symmetric
    lt = D.back_transform(L2)
    assert np.abs(lt - np.transpose(lt, (1, 0, 3, 2))).max() <= 1e-15 * np.abs(lt).max()


def test_linear_in_the_left_state():
    no, nv = 3, 5
    inp = make_inputs(no, nv, seed=4)
    A1, A2 = _left(no, nv, seed=5)
    B1, B2 = _left(no, nv, seed=6)
    ra, rb = _density(inp, 0.2, A1, A2), _density(inp, 0.2, B1, B2)
    rs = _density(inp, 0.2, 2.0 * A1 - B1, 2.0 * A2 - B2)
    for k in ("Doo", "Dov", "Dvv"):
        assert _rel(rs[k], 2.0 * ra[k] - rb[k]) < 1e-12


def test_flop_count():
    """6 nv^4 per distinct occupied permutation (tau3, X, Dvv) plus 24 nv no^3
    per virtual triple a >= b >= c (not all equal): 10 nv^4 no^3 to leading
    order."""
    no, nv = 4, 5
    inp = make_inputs(no, nv, seed=1)
    L1, L2 = _left(no, nv, seed=1)
    r = _density(inp, 0.0, L1, L2)
    nvt = nv * (nv + 1) * (nv + 2) // 6 - nv
    assert r["flops"] == 6 * nv ** 4 * (no ** 3 - no) + 24 * nv * no ** 3 * nvt


# ---- GPU: the library's FP64 density against the oracle -------------------------------------

@pytest.fixture(scope="module")
def g():
    import paper_2007_01088_gb300 as g
    return g


@pytest.mark.gpu
@pytest.mark.parametrize("no,nv", [(3, 9), (4, 20), (2, 17), (5, 33), (6, 24)])
def test_density_matches_oracle(g, no, nv):
    inp = make_inputs(no, nv, seed=300 + no * nv)
    L1, L2 = _left(no, nv, seed=no + 2 * nv)
    ctx = g.Context(inp)
    for w in (0.25, 0.0):
        ref = _density(inp, w, L1, L2)
        doo, dov, dvv = ctx.density(L1, L2, w)
        assert _rel(doo, ref["Doo"]) < 1e-11, ("Doo", w)
        assert _rel(dov, ref["Dov"]) < 1e-11, ("Dov", w)
        assert _rel(dvv, ref["Dvv"]) < 1e-11, ("Dvv", w)
    c = ctx.counters()
    nvt = nv * (nv + 1) * (nv + 2) // 6 - nv
    assert c["nominal_flop"] == 6 * nv ** 4 * (no ** 3 - no) + 24 * nv * no ** 3 * nvt
    assert c["launches"] > 0


@pytest.mark.gpu
def test_density_larger_shape(g):
    """Several W-build batches, multi-slab and single-slab virtual groups."""
    no, nv = 8, 64
    inp = make_inputs(no, nv, seed=11)
    L1, L2 = _left(no, nv, seed=12)
    ref = _density(inp, 0.1, L1, L2)
    doo, dov, dvv = g.Context(inp).density(L1, L2, 0.1)
    for x, k in ((doo, "Doo"), (dov, "Dov"), (dvv, "Dvv")):
        assert _rel(x, ref[k]) < 1e-11, k


@pytest.mark.gpu
def test_density_device_pointers(g):
    torch = pytest.importorskip("torch")
    no, nv = 4, 16
    inp = make_inputs(no, nv, seed=13)
    L1, L2 = _left(no, nv, seed=14)
    ref = _density(inp, 0.2, L1, L2)
    ctx = g.Context(inp, device=True)
    doo, dov, dvv = ctx.density(torch.from_numpy(L1).cuda(), torch.from_numpy(L2).cuda(), 0.2)
    for x, k in ((doo, "Doo"), (dov, "Dov"), (dvv, "Dvv")):
        assert _rel(x.cpu().numpy(), ref[k]) < 1e-11, k


@pytest.mark.gpu
def test_density_refusals(g):
    no, nv = 3, 8
    inp = make_inputs(no, nv, seed=15)
    L1, L2 = _left(no, nv, seed=16)
    ctx = g.Context(inp)

    def status(fn):
        with pytest.raises(g.CC3Error) as e:
            fn()
        return str(e.value)

    assert "(-7)" in status(lambda: ctx.density(L1, L2, 0.1, prec=g.CC3_SPLIT_INT8))
    # a frequency on a triples denominator (i = j = k included)
    eps = inp.eps_v[0] * 3 - inp.eps_o[0] * 3
    assert "(-5)" in status(lambda: ctx.density(L1, L2, float(eps)))
    assert "(-1)" in status(lambda: ctx.density(L1, L2, float("nan")))
    ctx.set_triples([[2, 1, 0]])
    assert "(-7)" in status(lambda: ctx.density(L1, L2, 0.1))
    assert "(-7)" in status(lambda: ctx.density(L1, L2, 0.1, prec=g.CC3_SPLIT_BF16))


@pytest.mark.gpu
@pytest.mark.parametrize("no,nv", [(2, 5), (7, 16)])
def test_density_small_and_ragged(g, no, nv):
    """no = 2 (two triples, each with one pair of equal indices) and a ragged shape
    with several occupied batches and 16 virtual slabs."""
    inp = make_inputs(no, nv, seed=no * 100 + nv)
    L1, L2 = _left(no, nv, seed=nv)
    ref = _density(inp, -0.15, L1, L2)
    doo, dov, dvv = g.Context(inp).density(L1, L2, -0.15)
    for x, k in ((doo, "Doo"), (dov, "Dov"), (dvv, "Dvv")):
        assert _rel(x, ref[k]) < 1e-11, k


# ---- split (BF16 slice) path -------------------------------------------------------------
# Left state normalised like the trial vectors, so that the absolute targets of
# the split path apply as for rho.

def _left_unit(no, nv, seed):
    L1, L2 = make_trial_vectors(no, nv, 1, seed=seed)
    return L1[0], L2[0]


@pytest.mark.gpu
@pytest.mark.parametrize("no,nv", [(3, 9), (4, 20), (2, 17), (5, 33), (6, 24), (7, 16)])
def test_split_density_matches_oracle(g, no, nv):
    inp = make_inputs(no, nv, seed=700 + no * nv)
    L1, L2 = _left_unit(no, nv, seed=no + 5 * nv)
    ctx = g.Context(inp)
    for w in (0.25, 0.0):
        ref = _density(inp, w, L1, L2)
        doo, dov, dvv = ctx.density(L1, L2, w, prec=g.CC3_SPLIT_BF16)
        for x, k in ((doo, "Doo"), (dov, "Dov"), (dvv, "Dvv")):
            assert split_close(x, ref[k]), (k, w, split_err(x, ref[k]))
    c = ctx.counters()
    nvt = nv * (nv + 1) * (nv + 2) // 6 - nv
    assert c["nominal_flop"] == 6 * nv ** 4 * (no ** 3 - no) + 24 * nv * no ** 3 * nvt
    assert c["slices"] == 6 and c["launches"] > 0
    # FP64 after split on the same context
    doo, dov, dvv = ctx.density(L1, L2, 0.0)
    for x, k in ((doo, "Doo"), (dov, "Dov"), (dvv, "Dvv")):
        assert _rel(x, ref[k]) < 1e-11, k


@pytest.mark.gpu
def test_split_density_larger_shape_and_device_pointers(g):
    """Several triple batches, device pointers and an odd nv."""
    torch = pytest.importorskip("torch")
    no, nv = 9, 37
    inp = make_inputs(no, nv, seed=21)
    L1, L2 = _left_unit(no, nv, seed=22)
    ref = _density(inp, -0.1, L1, L2)
    ctx = g.Context(inp, device=True)
    doo, dov, dvv = ctx.density(torch.from_numpy(L1).cuda(), torch.from_numpy(L2).cuda(),
                                -0.1, prec=g.CC3_SPLIT_BF16)
    for x, k in ((doo, "Doo"), (dov, "Dov"), (dvv, "Dvv")):
        x = x.cpu().numpy()
        assert split_close(x, ref[k]), (k, split_err(x, ref[k]))


@pytest.mark.gpu
def test_split_density_small(g):
    """no = 2: two triples with one pair of equal indices each, plus the
    i = j = k triples that only the resident D_oo term uses."""
    no, nv = 2, 5
    inp = make_inputs(no, nv, seed=23)
    L1, L2 = _left_unit(no, nv, seed=24)
    ref = _density(inp, 0.3, L1, L2)
    doo, dov, dvv = g.Context(inp).density(L1, L2, 0.3, prec=g.CC3_SPLIT_BF16)
    for x, k in ((doo, "Doo"), (dov, "Dov"), (dvv, "Dvv")):
        assert split_close(x, ref[k]), (k, split_err(x, ref[k]))


@pytest.mark.gpu
@pytest.mark.parametrize("no,nv", [(18, 10), (34, 6)])
def test_split_density_many_occupied(g, no, nv):
    """More than 16 occupied orbitals: each thread of the D_oo pair kernel sums
    several of the no^2 products, and at no = 34 a second group of 1024 products
    runs (the FP64 path stops at 24 occupied orbitals)."""
    inp = make_inputs(no, nv, seed=40 + no)
    L1, L2 = _left_unit(no, nv, seed=41 + no)
    ref = _density(inp, 0.2, L1, L2)
    doo, dov, dvv = g.Context(inp).density(L1, L2, 0.2, prec=g.CC3_SPLIT_BF16)
    for x, k in ((doo, "Doo"), (dov, "Dov"), (dvv, "Dvv")):
        assert split_close(x, ref[k]), (k, split_err(x, ref[k]))


@pytest.mark.gpu
def test_density_single_occupied_is_zero(g):
    """no = 1: every occupied triple has i = j = k, so tau~ and L3~ vanish and
    all three blocks are zero on both paths (the split path still builds tau3
    and L3 of the one triple for its D_oo pairs)."""
    inp = make_inputs(1, 7, seed=5)
    L1, L2 = _left_unit(1, 7, seed=6)
    ctx = g.Context(inp)
    for prec in (g.CC3_FP64, g.CC3_SPLIT_BF16):
        for x in ctx.density(L1, L2, 0.1, prec=prec):
            assert np.abs(np.asarray(x)).max() < 1e-30, prec
