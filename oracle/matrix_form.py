"""The restricted triple loop with library matrix products as its steps --
TEST INFRASTRUCTURE ONLY (see the package docstring).

The same steps as the C oracle (Algorithm 1 of arXiv 2007.01088 and the right
Jacobian transformation reconstructed from eq. "jcc3"), in the paper's order,
for one occupied triple i >= j >= k at a time, but each contraction is one
numpy tensor product (a BLAS matrix multiply) and each index permutation a
numpy transpose.  It exists because the plain C loops need minutes per triple
at nv ~ 200, the size of the batched-Jacobian workload, while these products
take a fraction of a second; it is pinned to the C oracle on small inputs
(general non-symmetric blocks, triple subsets, non-zero frequencies) in
``tests/test_oracle_pins.py``.

Conventions are those of the C oracle:
  B_pqr[x][y][z] = sum_d t[p][q][x][d] g_vvvo[y][d][z][r]
                 - sum_l t[p][l][x][y] g_oovo[l][q][z][r]
  W = P^{abc}_{ijk} B (six terms; term s places B of the ordered triple
      (ijk[s0], ijk[s1], ijk[s2]) with virtual index v[s_k] in its slot k)
  tau = W / (w - eps), eps^{abc}_{ijk} = e_a + e_b + e_c - e_i - e_j - e_k
  tau~ = 4 tau^{abc} - 2 tau^{acb} - 2 tau^{cba} - 2 tau^{bac} + tau^{bca} + tau^{cab}
  for each distinct ordered (p,q,r) with slot map m, V = tau~ viewed with
  x in slot m0, y in m1, z in m2:
    Omega1[p][x]       += sum_yz V[x][y][z] g_ovov[q][y][r][z]
    Omega~[p][q][x][y] += sum_z  V[x][y][z] F[r][z]
    Omega~[p][l][x][y] -= sum_z  V[x][y][z] g_ooov[q][l][r][z]
    Omega~[p][q][x][d] += sum_yz V[x][y][z] g_vvov[d][y][r][z]
  Omega2 = (1/3) P^{ab}_{ij} (2 Omega~ + Omega~^{ba}),  E_T = sum t2 Omega~.
"""
from __future__ import annotations

import numpy as np

# the six terms of P^{abc}_{ijk}, in the order of eq. "permutation"
PERM6 = ((0, 1, 2), (1, 0, 2), (2, 1, 0), (0, 2, 1), (1, 2, 0), (2, 0, 1))


def all_triples(no):
    return [(i, j, k) for i in range(no) for j in range(i + 1) for k in range(j + 1)
            if not (i == j == k)]


def distinct_perms(ijk):
    """Slot maps m of the distinct ordered triples (ijk[m0], ijk[m1], ijk[m2])."""
    if ijk[0] == ijk[1] == ijk[2]:
        return []
    seen, out = set(), []
    for m in PERM6:
        key = (ijk[m[0]], ijk[m[1]], ijk[m[2]])
        if key not in seen:
            seen.add(key)
            out.append(m)
    return out


class Blocks(dict):
    """The integral blocks, plus copies with the occupied index r outermost
    (vvvo as [r][d][y][z], vvov as [r][d][y][z]) so that each per-triple
    product reads one contiguous matrix."""

    def __init__(self, b):
        super().__init__(b)
        self.vvvo_r = np.ascontiguousarray(np.transpose(b["vvvo"], (3, 1, 0, 2)))
        self.vvov_r = np.ascontiguousarray(np.transpose(b["vvov"], (2, 0, 1, 3)))


def build_B(t, vvvo_r, oovo, p, q, r):
    """B_pqr[x][y][z] (one matrix product for each of the two sums);
    vvvo_r[r][d][y][z] = g_vvvo[y][d][z][r]."""
    nv = t.shape[2]
    vir = (t[p, q] @ vvvo_r[r].reshape(nv, nv * nv)).reshape(nv, nv, nv)   # (x, y, z)
    occ = np.tensordot(t[p], oovo[:, q, :, r], axes=([0], [0]))            # (x, y, z)
    return vir - occ


def build_W(t, vvvo_r, oovo, ijk):
    """W = P^{abc}_{ijk} B: W[v0][v1][v2] += B_(ijk[m]) [v[m0]][v[m1]][v[m2]]."""
    cache = {}
    W = None
    for m in PERM6:
        key = (ijk[m[0]], ijk[m[1]], ijk[m[2]])
        if key not in cache:
            cache[key] = build_B(t, vvvo_r, oovo, *key)
        term = np.transpose(cache[key], np.argsort(m))
        W = term.copy() if W is None else W + term
    return W


def divide(W, eps_o, eps_v, ijk, w):
    ev = np.asarray(eps_v)
    e = (ev[:, None, None] + ev[None, :, None] + ev[None, None, :]
         - (eps_o[ijk[0]] + eps_o[ijk[1]] + eps_o[ijk[2]]))
    return W / (w - e)


def contravariant(tau):
    return (4.0 * tau - 2.0 * tau.transpose(0, 2, 1) - 2.0 * tau.transpose(2, 1, 0)
            - 2.0 * tau.transpose(1, 0, 2) + tau.transpose(2, 0, 1) + tau.transpose(1, 2, 0))


def contract(V, blocks, p, q, r, om1, omt):
    """The four contractions of one ordered triple (p,q,r) into om1, omt."""
    nv = V.shape[0]
    Vm = V.reshape(nv, nv * nv)                                          # (x, (y, z))
    om1[p] += Vm @ blocks["ovov"][q, :, r, :].reshape(nv * nv)
    omt[p, q] += V @ blocks["F_ov"][r]
    omt[p] -= np.tensordot(V, blocks["ooov"][q, :, r, :], axes=([2], [1])).transpose(2, 0, 1)
    omt[p, q] += Vm @ blocks.vvov_r[r].reshape(nv, nv * nv).T


def loop(no, nv, tt_of, blocks, triples, om1, omt):
    """Runs the contractions of tau~ = tt_of(ijk) for every triple."""
    for ijk in triples:
        maps = distinct_perms(ijk)
        if not maps:
            continue
        tt = tt_of(ijk)
        for m in maps:
            contract(np.ascontiguousarray(tt.transpose(m)), blocks,
                     ijk[m[0]], ijk[m[1]], ijk[m[2]], om1, omt)


def back_transform(omt):
    x = (2.0 * omt + omt.transpose(0, 1, 3, 2)) / 3.0
    return x + x.transpose(1, 0, 3, 2)


def omega(no, nv, eps_o, eps_v, t2, blocks, triples=None):
    """Algorithm 1 on the general five blocks (dict vvvo, oovo, ooov, ovov,
    vvov, F_ov).  Returns dict(omega1, omega2, omega2_tilde, E_T)."""
    triples = all_triples(no) if triples is None else [tuple(int(x) for x in t) for t in triples]
    eo = np.asarray(eps_o)
    blocks = blocks if isinstance(blocks, Blocks) else Blocks(blocks)
    om1 = np.zeros((no, nv))
    omt = np.zeros((no, no, nv, nv))

    def tt_of(ijk):
        W = build_W(t2, blocks.vvvo_r, blocks["oovo"], ijk)
        return contravariant(divide(W, eo, eps_v, ijk, 0.0))

    loop(no, nv, tt_of, blocks, triples, om1, omt)
    return dict(omega1=om1, omega2=back_transform(omt), omega2_tilde=omt,
                E_T=float(np.sum(t2 * omt)))


def integral_blocks(no, nv, L):
    """(pq|rs) = sum_J L^J_pq L^J_rs for the ovvo, vvoo, oooo, oovv and ovov
    kinds, and the vv block of the Cholesky vectors."""
    o, v = slice(0, no), slice(no, no + nv)

    def blk(p, q, r, s):
        A, B = L[:, p, q], L[:, r, s]
        return np.tensordot(A, B, axes=([0], [0]))

    return dict(ovvo=blk(o, v, v, o), vvoo=blk(v, v, o, o), oooo=blk(o, o, o, o),
                oovv=blk(o, o, v, v), ovov=blk(o, v, o, v),
                Lvv=np.ascontiguousarray(L[:, v, v]))


def dressed_blocks(no, nv, L, R1, ib=None):
    """The R1-dressed blocks of the first-order T1 transformation, as in the C
    oracle: g^_bdck, g^_ljck, g^_jlkc, g^_dbkc and F^_kc (vvvv through the
    Cholesky vectors).  ib: integral_blocks(no, nv, L), if already formed."""
    ib = integral_blocks(no, nv, L) if ib is None else ib
    ovvo, vvoo, oooo, oovv, ovov = (ib[k] for k in ("ovvo", "vvoo", "oooo", "oovv", "ovov"))
    Lvv = ib["Lvv"]
    R = np.asarray(R1)
    M = np.tensordot(Lvv, R, axes=([2], [1]))                            # M[J][c][k]
    hvvvo = (-np.tensordot(R, ovvo, axes=([0], [0]))                      # (b, d, c, k)
             - np.tensordot(vvoo, R, axes=([2], [0])).transpose(0, 1, 3, 2)
             + np.tensordot(Lvv, M, axes=([0], [0])))
    hoovo = (np.tensordot(R, ovvo, axes=([1], [1])).transpose(1, 0, 2, 3)   # (l, j, c, k)
             - np.tensordot(oooo, R, axes=([2], [0])).transpose(0, 1, 3, 2)
             + np.tensordot(oovv, R, axes=([3], [1])))
    hooov = np.tensordot(ovov, R, axes=([1], [1])).transpose(0, 3, 1, 2)   # (j, l, k, c)
    hvvov = -np.tensordot(R, ovov, axes=([0], [0]))                       # (d, b, k, c)
    hF = 2.0 * np.tensordot(ovov, R, axes=([2, 3], [0, 1])) \
        - np.tensordot(ovov.transpose(0, 3, 2, 1), R, axes=([2, 3], [0, 1]))
    return dict(vvvo=hvvvo, oovo=hoovo, ooov=hooov, vvov=hvvov, F_ov=hF)


def jacobian(inp, R1, R2, w, triples=None, blocks=None):
    """Right Jacobian transformation of trial vectors R1[n], R2[n] at
    frequencies w[n] on a cc3_inputs problem (symmetric blocks).  Returns
    dict(rho1, rho2)."""
    from . import symmetric_blocks
    no, nv = inp.no, inp.nv
    g = Blocks(symmetric_blocks(inp) if blocks is None else blocks)
    R1 = np.asarray(R1).reshape(-1, no, nv)
    nvec = R1.shape[0]
    R2 = np.asarray(R2).reshape(nvec, no, no, nv, nv)
    w = np.broadcast_to(np.asarray(w, dtype=np.float64), (nvec,))
    triples = all_triples(no) if triples is None else [tuple(int(x) for x in t) for t in triples]
    eo, ev, t2 = np.asarray(inp.eps_o), np.asarray(inp.eps_v), np.asarray(inp.t2)
    L = np.asarray(inp.chol_L)
    rho1 = np.zeros((nvec, no, nv))
    rho2 = np.zeros((nvec, no, no, nv, nv))
    # tau~3 of every triple (shared by the vectors)
    tau_tt = {}
    for ijk in triples:
        if distinct_perms(ijk):
            W = build_W(t2, g.vvvo_r, g["oovo"], ijk)
            tau_tt[ijk] = contravariant(divide(W, eo, ev, ijk, 0.0))
    ib = integral_blocks(no, nv, L)
    for n in range(nvec):
        h = dressed_blocks(no, nv, L, R1[n], ib)
        hb = Blocks(dict(vvvo=h["vvvo"], oovo=h["oovo"], ooov=h["ooov"], vvov=h["vvov"],
                         ovov=np.zeros_like(g["ovov"]), F_ov=h["F_ov"]))
        om1 = np.zeros((no, nv))
        omt = np.zeros((no, no, nv, nv))

        def r3_tt(ijk):
            W = build_W(R2[n], g.vvvo_r, g["oovo"], ijk) + build_W(t2, hb.vvvo_r, h["oovo"], ijk)
            return contravariant(divide(W, eo, ev, ijk, w[n]))

        loop(no, nv, r3_tt, g, triples, om1, omt)
        loop(no, nv, lambda ijk: tau_tt[ijk], hb, triples, om1, omt)
        rho1[n] = om1
        rho2[n] = back_transform(omt)
    return dict(rho1=rho1, rho2=rho2)


def left_jacobian(inp, L1, L2, w, triples=None):
    """Left (transpose) Jacobian transformation, the steps of the C oracle's
    oracle_left_jacobian with numpy products (symmetric blocks).  Returns
    dict(sigma1, sigma2)."""
    from . import symmetric_blocks
    no, nv = inp.no, inp.nv
    g = Blocks(symmetric_blocks(inp))
    L1 = np.asarray(L1).reshape(-1, no, nv)
    nvec = L1.shape[0]
    L2 = np.asarray(L2).reshape(nvec, no, no, nv, nv)
    w = np.broadcast_to(np.asarray(w, dtype=np.float64), (nvec,))
    triples = all_triples(no) if triples is None else [tuple(int(x) for x in t) for t in triples]
    eo, ev, t2 = np.asarray(inp.eps_o), np.asarray(inp.eps_v), np.asarray(inp.t2)
    L = np.asarray(inp.chol_L)
    ib = integral_blocks(no, nv, L)
    ovov, vvoo, oooo, oovv = ib["ovov"], ib["vvoo"], ib["oooo"], ib["oovv"]
    ovvo = ib["ovvo"]
    vvov_r = g.vvov_r                               # [r][d][y][z] = g_dyrz
    ooov = g["ooov"]
    tau_tt = {}
    for ijk in triples:
        if distinct_perms(ijk):
            W = build_W(t2, g.vvvo_r, g["oovo"], ijk)
            tau_tt[ijk] = contravariant(divide(W, eo, ev, ijk, 0.0))
    s1 = np.zeros((nvec, no, nv))
    s2 = np.zeros((nvec, no, no, nv, nv))
    for n in range(nvec):
        l1 = L1[n]
        lt = back_transform(L2[n])                 # the back-transform is symmetric
        sig1 = np.zeros((no, nv))
        sig2 = np.zeros((no, no, nv, nv))
        Q = np.zeros((no, nv))
        G = np.zeros((nv, nv, nv, no))             # [y][d][z][r]
        H = np.zeros((no, no, nv, no))             # [l][q][z][r]
        for ijk in triples:
            maps = distinct_perms(ijk)
            if not maps:
                continue
            tt = tau_tt[ijk]
            for m in maps:
                p, q, r = ijk[m[0]], ijk[m[1]], ijk[m[2]]
                V = np.ascontiguousarray(tt.transpose(m))
                Q[r] += np.tensordot(lt[p, q], V, axes=([0, 1], [0, 1]))
                # - sum_xyz Lt[p][l][x][y] V[x][y][z] (qd|rz)
                T = V @ ovov[q, :, r, :].T                                   # (x, y, d)
                sig1 -= np.tensordot(lt[p], T, axes=([1, 2], [0, 1]))       # (l, d)
                # - sum_xyz Lt[p][q][x][d] V[x][y][z] (ly|rz)
                U = np.tensordot(V, ovov[:, :, r, :], axes=([1, 2], [1, 2]))  # (x, l)
                sig1 -= U.T @ lt[p, q]
            # L3 numerator, P X
            cache = {}
            X = None
            for m in PERM6:
                key = (ijk[m[0]], ijk[m[1]], ijk[m[2]])
                if key not in cache:
                    p, q, r = key
                    B = (l1[p][:, None, None] * ovov[q, :, r, :][None, :, :]
                         + lt[p, q][:, :, None] * g["F_ov"][r][None, None, :])
                    B = B + (lt[p, q] @ vvov_r[r].reshape(nv, nv * nv)).reshape(nv, nv, nv)
                    B = B - np.tensordot(lt[p], ooov[q, :, r, :], axes=([0], [0]))
                    cache[key] = B
                term = np.transpose(cache[key], np.argsort(m))
                X = term.copy() if X is None else X + term
            Vt = contravariant(divide(X, eo, ev, ijk, w[n]))
            for m in maps:
                p, q, r = ijk[m[0]], ijk[m[1]], ijk[m[2]]
                V = np.ascontiguousarray(Vt.transpose(m))
                Vm = V.reshape(nv, nv * nv)
                # sigma2[p][q][x][d] += sum_yz V g_{ydzr};  g_ydzr = vvvo_r[r][d][y][z]
                sig2[p, q] += Vm @ g.vvvo_r[r].reshape(nv, nv * nv).T
                # sigma2[p][l][x][y] -= sum_z V g_{lqzr}
                sig2[p] -= np.tensordot(V, g["oovo"][:, q, :, r], axes=([2], [1])).transpose(2, 0, 1)
                # G[y][d][z][r] += sum_x V[x][y][z] t[p][q][x][d]
                G[:, :, :, r] += np.tensordot(V, t2[p, q], axes=([0], [0])).transpose(0, 2, 1)
                # H[l][q][z][r] += sum_xy V[x][y][z] t[p][l][x][y]
                H[:, q, :, r] += np.tensordot(t2[p], V, axes=([1, 2], [0, 1]))
        sig1 += 2.0 * np.tensordot(Q, ovov, axes=([0, 1], [0, 1])) \
            - np.tensordot(Q, ovov.transpose(0, 3, 2, 1), axes=([0, 1], [0, 1]))
        sig1 -= np.tensordot(ovvo, G, axes=([1, 2, 3], [1, 2, 3]))                # (l, b)
        sig1 -= np.tensordot(vvoo, G, axes=([0, 1, 3], [0, 1, 3]))                 # (l, c)
        N = np.tensordot(ib["Lvv"], G, axes=([1, 2], [0, 1]))                       # (J, c, k)
        sig1 += np.tensordot(N, ib["Lvv"], axes=([0, 1], [0, 1]))                   # (k, e)
        sig1 -= np.tensordot(H, ovvo, axes=([0, 2, 3], [0, 2, 3]))                 # (j, d)
        sig1 += np.tensordot(oooo, H, axes=([0, 1, 3], [0, 1, 3]))                 # (m, c)
        sig1 -= np.tensordot(H, oovv, axes=([0, 1, 2], [0, 1, 2]))                 # (k, d)
        s1[n] = sig1
        s2[n] = 0.5 * (sig2 + sig2.transpose(1, 0, 3, 2))
    return dict(sigma1=s1, sigma2=s2)
