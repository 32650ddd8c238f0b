"""Pins of the FP64 oracle against what the paper and the mathematics fix
(arXiv 2007.01088; Algorithm 1, eq. "permutation", the six-fold symmetry,
the permutation count rule, the contravariant transformation, eq. "jcc3").

No GPU.  The restricted-loop C oracle is checked against the full-tensor
definition, against symmetry and scaling laws, against the printed FLOP counts,
against two closed-form energy identities, and (Jacobian) against the exact
derivative of the residual through the T1 transformation."""
import os

import numpy as np
import pytest

import oracle
from oracle import definition as D
from cc3_inputs import make_inputs, make_trial_vectors, unique_triples

HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    s = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() / s


@pytest.fixture(scope="module")
def cfg1():
    return make_inputs(5, 30, 0)


# --- P1: the restricted loop equals the full-tensor definition -------------
@pytest.mark.parametrize("no,nv", [(2, 5), (3, 4), (4, 7), (5, 30)])
def test_restricted_loop_equals_full_tensor(no, nv):
    inp = make_inputs(no, nv, 0)
    b = oracle.symmetric_blocks(inp)
    r1 = oracle.omega_inputs(inp)
    r2 = D.omega_full(inp.eps_o, inp.eps_v, inp.t2, b)
    assert rel(r1["omega1"], r2["omega1"]) < 1e-13
    assert rel(r1["omega2"], r2["omega2"]) < 1e-13
    assert rel(r1["omega2_tilde"], r2["omega2_tilde"]) < 1e-13
    assert abs(r1["E_T"] - r2["E_T"]) <= 1e-13 * abs(r2["E_T"])


def test_no1_gives_zero():
    # no = 1: every triple has i = j = k, which contributes nothing
    inp = make_inputs(1, 6, 0)
    r = oracle.omega_inputs(inp)
    assert np.all(r["omega1"] == 0) and np.all(r["omega2"] == 0) and r["E_T"] == 0.0


def test_general_blocks_nonsymmetric():
    # T1-transformed integrals lack pq<->qp symmetry; the restricted loop must
    # still equal the definition term by term
    inp = make_inputs(3, 6, 2)
    t1 = np.random.default_rng(9).normal(0, 0.2, size=(3, 6))
    b = oracle.t1_transform(inp, t1)
    assert np.abs(b["vvvo"] - np.transpose(b["vvov"], (1, 0, 3, 2))).max() > 1e-4
    r1 = oracle.omega(3, 6, inp.eps_o, inp.eps_v, inp.t2, b)
    r2 = D.omega_full(inp.eps_o, inp.eps_v, inp.t2, b)
    assert rel(r1["omega1"], r2["omega1"]) < 1e-13
    assert rel(r1["omega2"], r2["omega2"]) < 1e-13


def test_triple_subsets_are_additive(cfg1):
    tr = [t[:3] for t in unique_triples(cfg1.no)]
    full = oracle.omega_inputs(cfg1)
    a = oracle.omega_inputs(cfg1, triples=tr[::2])
    b = oracle.omega_inputs(cfg1, triples=tr[1::2])
    assert rel(a["omega2"] + b["omega2"], full["omega2"]) < 1e-13
    assert abs(a["E_T"] + b["E_T"] - full["E_T"]) < 1e-13 * abs(full["E_T"])


# --- P2: symmetries ---------------------------------------------------------
def test_six_fold_symmetry_and_contravariant_diagonal():
    inp = make_inputs(4, 6, 1)
    b = oracle.symmetric_blocks(inp)
    r = D.omega_full(inp.eps_o, inp.eps_v, inp.t2, b)
    W, tau, tt = r["W"], r["tau"], r["tau_tilde"]
    E = np.einsum
    for spec in ["jikbac", "kjicba", "ikjacb", "jkibca", "kijcab"]:
        assert np.abs(E(spec + "->ijkabc", W) - W).max() < 1e-15 * np.abs(W).max() * 10
        assert np.abs(E(spec + "->ijkabc", tt) - tt).max() < 1e-14 * np.abs(tt).max()
    for i in range(inp.no):
        assert np.abs(tt[i, i, i]).max() < 1e-14 * np.abs(tt).max()
    # tau~^{aaa}_{ijk} = 0 (4-2-2-2+1+1 = 0)
    a = np.arange(inp.nv)
    assert np.abs(tt[:, :, :, a, a, a]).max() < 1e-14 * np.abs(tt).max()
    om2 = r["omega2"]
    assert np.abs(om2 - np.transpose(om2, (1, 0, 3, 2))).max() == 0.0


def test_permutation_counts():
    # 6 distinct permutations if i, j, k differ, 3 if two are equal, none if
    # all equal; the weights sum to the number of ordered triples minus no
    for no in range(1, 9):
        tr = unique_triples(no)
        assert sum(w for *_, w in tr) == no ** 3 - no
        assert all((w == 6) == (len({i, j, k}) == 3) for i, j, k, w in tr)


# --- P3: vanishing inputs ---------------------------------------------------
def test_zero_integrals_give_zero(cfg1):
    b = oracle.symmetric_blocks(cfg1)
    b0 = dict(b, vvvo=np.zeros_like(b["vvvo"]), oovo=np.zeros_like(b["oovo"]))
    r = oracle.omega(cfg1.no, cfg1.nv, cfg1.eps_o, cfg1.eps_v, cfg1.t2, b0)
    assert np.all(r["omega1"] == 0) and np.all(r["omega2"] == 0) and r["E_T"] == 0
    b1 = dict(b, F_ov=np.zeros_like(b["F_ov"]), ovov=np.zeros_like(b["ovov"]),
              ooov=np.zeros_like(b["ooov"]), vvov=np.zeros_like(b["vvov"]))
    r = oracle.omega(cfg1.no, cfg1.nv, cfg1.eps_o, cfg1.eps_v, cfg1.t2, b1)
    assert np.all(r["omega1"] == 0) and np.all(r["omega2"] == 0) and r["E_T"] == 0


# --- P4: FLOP counts --------------------------------------------------------
@pytest.mark.parametrize("no,nv", [(2, 3), (3, 4), (5, 6)])
def test_flop_count(no, nv):
    inp = make_inputs(no, nv, 0)
    assert oracle.omega_inputs(inp)["flops"] == 4 * nv ** 4 * (no ** 3 - no)
    assert oracle.prep(inp)["flops"] == 4 * nv ** 4 * (no ** 3 - no)


def test_flop_convention_reproduces_paper_table4():
    # efficiency = FLOP / (time * peak) with FLOP = m * nv^4 no^3 reproduces
    # the printed efficiencies (rounded to 0.1 %)
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "paper_table4_efficiency.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 7
    nv, no, peak = 544, 23, 2956.8e9
    for name, minutes, eff, mult in rows:
        flop = int(mult) * nv ** 4 * no ** 3
        e = 100.0 * flop / (float(minutes) * 60.0 * peak)
        assert abs(e - float(eff)) < 0.1, (name, e, eff)


# --- P5: closed-form energy identities -------------------------------------
def test_energy_identities():
    inp = make_inputs(4, 7, 3)
    b = oracle.symmetric_blocks(inp)
    r = oracle.omega_inputs(inp)
    full = D.omega_full(inp.eps_o, inp.eps_v, inp.t2, b)
    eps = D.denominators(inp.eps_o, inp.eps_v)
    tau, tt = full["tau"], full["tau_tilde"]
    # E_T = -(1/6) sum eps tau~ tau + sum t^{ab}_{ij} tau~^{abc}_{ijk} F_kc
    e_closed = (-np.sum(eps * tt * tau) / 6.0
                + np.einsum("ijab,ijkabc,kc->", inp.t2, tt, inp.F_ov))
    assert abs(r["E_T"] - e_closed) < 1e-12 * abs(e_closed)
    # sum (2 t^{ab}_{ij} - t^{ba}_{ij}) Omega2^{ab}_{ij} = 2 E_T
    u = 2 * inp.t2 - np.transpose(inp.t2, (0, 1, 3, 2))
    assert abs(np.sum(u * r["omega2"]) - 2 * r["E_T"]) < 1e-12 * abs(r["E_T"])


# --- P6: scaling laws, covariant/contravariant round trip -------------------
def test_homogeneity(cfg1):
    b = oracle.symmetric_blocks(cfg1)
    base = oracle.omega_inputs(cfg1)
    r = oracle.omega(cfg1.no, cfg1.nv, cfg1.eps_o, cfg1.eps_v, 1.7 * cfg1.t2, b)
    assert rel(r["omega2"], 1.7 * base["omega2"]) < 1e-13
    r = oracle.omega(cfg1.no, cfg1.nv, 2.0 * cfg1.eps_o, 2.0 * cfg1.eps_v, cfg1.t2, b)
    assert rel(r["omega2"], base["omega2"] / 2.0) < 1e-13
    bb = {k: 0.5 * v for k, v in b.items()}
    r = oracle.omega(cfg1.no, cfg1.nv, cfg1.eps_o, cfg1.eps_v, cfg1.t2, bb)
    assert rel(r["omega2"], 0.25 * base["omega2"]) < 1e-13


def test_back_transform_inverts_contravariant():
    X = np.random.default_rng(0).normal(size=(3, 3, 4, 4))
    Y = 2 * X - np.transpose(X, (0, 1, 3, 2))           # covariant -> contravariant
    Z = (2 * Y + np.transpose(Y, (0, 1, 3, 2))) / 3.0   # the paper's inverse
    assert np.abs(Z - X).max() < 1e-14


# --- Algorithm 2 and the Jacobian -------------------------------------------
@pytest.fixture(scope="module")
def tiny():
    inp = make_inputs(3, 5, 0)
    R1, R2 = make_trial_vectors(3, 5, 2, seed=3)
    return inp, R1, R2


def test_dressed_blocks_are_the_t1_derivative(tiny):
    inp, R1, _ = tiny
    exact = D.t1_derivative_blocks(inp, R1[0])
    mine = oracle.dressed_blocks(inp, R1[0])
    for k, v in mine.items():
        assert np.abs(v - exact[k]).max() < 1e-14 * max(np.abs(exact[k]).max(), 1e-30), k
    assert np.abs(exact["ovov"]).max() == 0.0


def test_jacobian_is_derivative_of_residual(tiny):
    # J3: rho(R; w=0) = d/dh Omega_T(t1 = h R1, t2 + h R2) at h = 0, taken by
    # complex-step differentiation of the full-tensor residual
    inp, R1, R2 = tiny
    h = 1e-30
    for n in range(2):
        blk = oracle.t1_transform_complex(inp, 1j * h * R1[n])
        res = D.omega_full(inp.eps_o, inp.eps_v, inp.t2 + 1j * h * R2[n], blk)
        jac = oracle.jacobian(inp, R1[n:n + 1], R2[n:n + 1], [0.0])
        assert rel(jac["rho1"][0], np.imag(res["omega1"]) / h) < 1e-12
        assert rel(jac["rho2"][0], np.imag(res["omega2"]) / h) < 1e-12


def test_jacobian_restricted_equals_full_at_frequency(tiny):
    inp, R1, R2 = tiny
    b = oracle.symmetric_blocks(inp)
    w = [0.25, -0.1]
    jac = oracle.jacobian(inp, R1, R2, w)
    for n in range(2):
        db = D.t1_derivative_blocks(inp, R1[n])
        full = D.jacobian_full(inp, R1[n], R2[n], w[n], b, db)
        assert rel(jac["rho1"][n], full["rho1"]) < 1e-12
        assert rel(jac["rho2"][n], full["rho2"]) < 1e-12


def test_jacobian_on_t2_is_residual(tiny):
    # J1: w = 0, R1 = 0, R2 = t2 gives rho = Omega
    inp, _, _ = tiny
    jac = oracle.jacobian(inp, np.zeros((1, 3, 5)), inp.t2[None], [0.0])
    om = oracle.omega_inputs(inp)
    assert rel(jac["rho2"][0], om["omega2"]) < 1e-13
    assert rel(jac["rho1"][0], om["omega1"]) < 1e-13


def test_jacobian_linear(tiny):
    inp, R1, R2 = tiny
    a = oracle.jacobian(inp, R1[:1], R2[:1], [0.2])
    b = oracle.jacobian(inp, R1[1:], R2[1:], [0.2])
    c = oracle.jacobian(inp, 2 * R1[:1] - R1[1:], 2 * R2[:1] - R2[1:], [0.2])
    assert rel(c["rho2"][0], 2 * a["rho2"][0] - b["rho2"][0]) < 1e-12


def test_prep_intermediates_give_dressed_contractions(tiny):
    # Algorithm 2's Zv, Zo contracted with R1 equal the direct contractions of
    # tau~ with the dressed ooov and vvov blocks
    inp, R1, _ = tiny
    no, nv = inp.no, inp.nv
    b = oracle.symmetric_blocks(inp)
    full = D.omega_full(inp.eps_o, inp.eps_v, inp.t2, b)
    db = oracle.dressed_blocks(inp, R1[0])
    z = oracle.prep(inp)
    direct = (-np.einsum("ijkabc,jlkc->ilab", full["tau_tilde"], db["ooov"])
              + np.einsum("ijkabc,dbkc->ijad", full["tau_tilde"], db["vvov"]))
    via_z = (np.einsum("abid,ld->ilab", z["Zv"], R1[0])
             - np.einsum("ajil,ld->ijad", z["Zo"], R1[0]))
    assert rel(via_z, direct) < 1e-12


# --- the matrix-product form of the restricted loop -------------------------
# oracle.matrix_form takes the same steps with numpy tensor products; it serves
# the GPU tests at the batched-Jacobian shape (nv = 200), where the C loops take
# minutes per triple.  Pinned here to the C oracle (itself pinned above) on
# general non-symmetric blocks, triple subsets and non-zero frequencies.
def test_matrix_form_residual_equals_c_oracle():
    from oracle import matrix_form as MF
    inp = make_inputs(4, 7, 3)
    t1 = np.random.default_rng(4).normal(0, 0.2, size=(4, 7))
    b = oracle.t1_transform(inp, t1)
    tr = [t[:3] for t in unique_triples(4)]
    for sel in (None, tr[::3]):
        r1 = oracle.omega(4, 7, inp.eps_o, inp.eps_v, inp.t2, b, triples=sel)
        r2 = MF.omega(4, 7, inp.eps_o, inp.eps_v, inp.t2, b, triples=sel)
        for k in ("omega1", "omega2", "omega2_tilde"):
            assert rel(r2[k], r1[k]) < 1e-13, k
        assert abs(r2["E_T"] - r1["E_T"]) <= 1e-13 * abs(r1["E_T"])


def test_matrix_form_dressed_blocks_equal_c_oracle(tiny):
    from oracle import matrix_form as MF
    inp, R1, _ = tiny
    ref = oracle.dressed_blocks(inp, R1[1])
    mine = MF.dressed_blocks(inp.no, inp.nv, inp.chol_L, R1[1])
    for k, v in ref.items():
        assert rel(mine[k], v) < 1e-13, k


def test_matrix_form_jacobian_equals_c_oracle():
    from oracle import matrix_form as MF
    inp = make_inputs(4, 9, 6)
    R1, R2 = make_trial_vectors(4, 9, 3, seed=8)
    w = [0.25, 0.0, -0.1]
    tr = [t[:3] for t in unique_triples(4)]
    for sel in (None, [tr[1], tr[-1], tr[4]]):
        ref = oracle.jacobian(inp, R1, R2, w, triples=sel)
        mine = MF.jacobian(inp, R1, R2, w, triples=sel)
        assert rel(mine["rho1"], ref["rho1"]) < 1e-12
        assert rel(mine["rho2"], ref["rho2"]) < 1e-12


# --- left (transpose) Jacobian ------------------------------------------------
# The left transformation is read as the exact transpose of the right one under
# the plain inner product over the elements of (R1, R2) with pair-symmetric R2.
# It is pinned to the right Jacobian (itself pinned to the derivative of the
# residual above) through the bilinear identity sum L.rho(R) = sum sigma(L).R.
def _pair_sym(x):
    return 0.5 * (x + np.transpose(x, (0, 2, 1, 4, 3)))


def _left_vectors(no, nv, n, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, no, nv)), _pair_sym(rng.normal(size=(n, no, no, nv, nv)))


@pytest.mark.parametrize("no,nv", [(2, 5), (3, 4), (4, 7)])
def test_left_jacobian_is_the_transpose_of_the_right(no, nv):
    inp = make_inputs(no, nv, seed=no + nv)
    R1, R2 = make_trial_vectors(no, nv, 2, seed=3)
    L1, L2 = _left_vectors(no, nv, 2, seed=5)
    tr = [t[:3] for t in unique_triples(no)]
    for w, sel in [(0.0, None), (0.25, None), (-0.1, tr[::2])]:
        rho = oracle.jacobian(inp, R1, R2, [w, w], triples=sel)
        sig = oracle.left_jacobian(inp, L1, L2, [w, w], triples=sel)
        for n in range(2):
            for m in range(2):
                a = np.sum(L1[n] * rho["rho1"][m]) + np.sum(L2[n] * rho["rho2"][m])
                b = np.sum(sig["sigma1"][n] * R1[m]) + np.sum(sig["sigma2"][n] * R2[m])
                scale = (np.abs(L1[n]).sum() * np.abs(rho["rho1"][m]).max()
                         + np.abs(L2[n]).sum() * np.abs(rho["rho2"][m]).max())
                assert abs(a - b) <= 1e-13 * scale, (w, n, m, a, b)


def test_left_jacobian_matrix_equals_transposed_right_matrix():
    # every column of the right Jacobian (unit R) against every row of the left
    # one (unit L), on a two-orbital, three-virtual problem
    no, nv = 2, 3
    inp = make_inputs(no, nv, seed=4)
    n1 = no * nv
    basis = []  # unit vectors of (R1, pair-symmetric R2)
    for k in range(n1):
        e1 = np.zeros(n1)
        e1[k] = 1.0
        basis.append((e1.reshape(no, nv), np.zeros((no, no, nv, nv))))
    for i in range(no):
        for j in range(no):
            for a in range(nv):
                for b in range(nv):
                    if (i, a) <= (j, b):
                        e2 = np.zeros((no, no, nv, nv))
                        e2[i, j, a, b] = e2[j, i, b, a] = 1.0
                        basis.append((np.zeros((no, nv)), e2))
    R1 = np.stack([x[0] for x in basis])
    R2 = np.stack([x[1] for x in basis])
    w = [0.2] * len(basis)
    rho = oracle.jacobian(inp, R1, R2, w)
    sig = oracle.left_jacobian(inp, R1, R2, w)
    J = np.array([[np.sum(R1[n] * rho["rho1"][m]) + np.sum(R2[n] * rho["rho2"][m])
                   for m in range(len(basis))] for n in range(len(basis))])
    S = np.array([[np.sum(sig["sigma1"][n] * R1[m]) + np.sum(sig["sigma2"][n] * R2[m])
                   for m in range(len(basis))] for n in range(len(basis))])
    assert np.abs(J).max() > 1e-6
    assert np.abs(J - S).max() <= 1e-13 * np.abs(J).max()


def test_left_jacobian_linear_zero_symmetric_and_flops():
    no, nv = 3, 6
    inp = make_inputs(no, nv, seed=12)
    L1, L2 = _left_vectors(no, nv, 2, seed=1)
    a = oracle.left_jacobian(inp, L1[:1], L2[:1], [0.3])
    b = oracle.left_jacobian(inp, L1[1:], L2[1:], [0.3])
    c = oracle.left_jacobian(inp, 2 * L1[:1] - 3 * L1[1:], 2 * L2[:1] - 3 * L2[1:], [0.3])
    for k in ("sigma1", "sigma2"):
        assert rel(c[k][0], 2 * a[k][0] - 3 * b[k][0]) < 1e-12
    s2 = a["sigma2"][0]
    assert np.array_equal(s2, np.transpose(s2, (1, 0, 3, 2)))
    z = oracle.left_jacobian(inp, np.zeros((1, no, nv)), np.zeros((1, no, no, nv, nv)), [0.3])
    assert not z["sigma1"].any() and not z["sigma2"].any()
    # 8 nv^4 per distinct permutation: tau3, the L3 numerator, sigma2 and G
    assert a["flops"] == 8 * nv ** 4 * (no ** 3 - no)


def test_matrix_form_left_jacobian_equals_c_oracle():
    from oracle import matrix_form as MF
    inp = make_inputs(4, 9, 6)
    L1, L2 = _left_vectors(4, 9, 2, seed=9)
    w = [0.25, -0.1]
    tr = [t[:3] for t in unique_triples(4)]
    for sel in (None, [tr[1], tr[-1], tr[4]]):
        ref = oracle.left_jacobian(inp, L1, L2, w, triples=sel)
        mine = MF.left_jacobian(inp, L1, L2, w, triples=sel)
        assert rel(mine["sigma1"], ref["sigma1"]) < 1e-12
        assert rel(mine["sigma2"], ref["sigma2"]) < 1e-12
