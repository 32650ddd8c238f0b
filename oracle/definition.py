"""The CC3 triples residual by its plain definition over the full tensor --
TEST INFRASTRUCTURE ONLY (see the package docstring).

Every ordered occupied triple (i,j,k) is built as one nv^3 no^3 tensor, with no
restricted loop and no permutation bookkeeping: the restricted loop of
Algorithm 1 (arXiv 2007.01088) is an exact refactoring of these sums, which is
what the oracle's tests check.  Only for tiny sizes (memory nv^3 no^3).

  B^{abc}_{ijk} = sum_d t^{ad}_{ij} g_{bdck} - sum_l t^{ab}_{il} g_{ljck}
  W = P^{abc}_{ijk} B      (eq. "permutation", six terms)
  tau = -W / eps^{abc}_{ijk}
  tau~ = 4 tau^{abc} - 2 tau^{acb} - 2 tau^{cba} - 2 tau^{bac} + tau^{bca} + tau^{cab}
  Omega1_ia   = sum_{jkbc} tau~^{abc}_{ijk} g_{jbkc}
  Omega~_ijab = sum_{kc} tau~^{abc}_{ijk} F_kc            (F term)
  Omega~_ilab -= sum_{jkc} tau~^{abc}_{ijk} g_{jlkc}      (ooov term)
  Omega~_ijad += sum_{kbc} tau~^{abc}_{ijk} g_{dbkc}      (vvov term)
  Omega2_ijab = X_ijab + X_jiba,  X = (2 Omega~_ijab + Omega~_ijba) / 3
  E_T = sum t_ijab Omega~_ijab

The i = j = k entries need no special case: there the six-fold symmetry makes
every virtual permutation of tau equal, and tau~ vanishes identically.
"""
from __future__ import annotations

import numpy as np

E = np.einsum


def _scalar(x):
    return complex(x) if np.iscomplexobj(x) else float(x)


def denominators(eps_o, eps_v):
    eo, ev = np.asarray(eps_o), np.asarray(eps_v)
    return (ev[None, None, None, :, None, None] + ev[None, None, None, None, :, None]
            + ev[None, None, None, None, None, :] - eo[:, None, None, None, None, None]
            - eo[None, :, None, None, None, None] - eo[None, None, :, None, None, None])


def W_full(t2, vvvo, oovo):
    B = E("ijad,bdck->ijkabc", t2, vvvo) - E("ilab,ljck->ijkabc", t2, oovo)
    return (B + E("jikbac->ijkabc", B) + E("kjicba->ijkabc", B)
            + E("ikjacb->ijkabc", B) + E("jkibca->ijkabc", B)
            + E("kijcab->ijkabc", B))


def contravariant(tau):
    return (4 * tau - 2 * E("ijkacb->ijkabc", tau) - 2 * E("ijkcba->ijkabc", tau)
            - 2 * E("ijkbac->ijkabc", tau) + E("ijkbca->ijkabc", tau)
            + E("ijkcab->ijkabc", tau))


def contractions(tt, blocks):
    om1 = E("ijkabc,jbkc->ia", tt, blocks["ovov"])
    omt = (E("ijkabc,kc->ijab", tt, blocks["F_ov"])
           - E("ijkabc,jlkc->ilab", tt, blocks["ooov"])
           + E("ijkabc,dbkc->ijad", tt, blocks["vvov"]))
    return om1, omt


def back_transform(omt):
    X = (2 * omt + E("ijba->ijab", omt)) / 3.0
    return X + E("jiba->ijab", X)


def omega_full(eps_o, eps_v, t2, blocks, w=0.0):
    """Full-tensor residual; returns dict(omega1, omega2, omega2_tilde, E_T,
    W, tau, tau_tilde)."""
    W = W_full(t2, blocks["vvvo"], blocks["oovo"])
    tau = W / (w - denominators(eps_o, eps_v))
    tt = contravariant(tau)
    om1, omt = contractions(tt, blocks)
    return dict(omega1=om1, omega2=back_transform(omt), omega2_tilde=omt,
                E_T=_scalar(np.sum(t2 * omt)), W=W, tau=tau, tau_tilde=tt)


def t1_derivative_blocks(inp, R1, h=1e-30):
    """First derivative along T1 = R1 of the T1-transformed blocks and F_ov,
    by complex-step differentiation of the exact transformation (no
    subtractive cancellation, exact to rounding): d/dh g~(h R1) at h = 0."""
    from . import t1_transform_complex
    tr = t1_transform_complex(inp, 1j * h * np.asarray(R1))
    return {k: np.imag(v) / h for k, v in tr.items()}


def jacobian_full(inp, R1, R2, w, blocks, dblocks):
    """Right Jacobian transformation by its full-tensor definition:
    R3 = [P(R2, g) + P(t2, g^)] / (w - eps), rho~ = contractions(R~3; g, F)
    + contractions(tau~; g^, F^), back-transformed as the residual.  dblocks
    are the dressed blocks (g^, F^), ovov^ = 0."""
    t2 = inp.t2
    WR = W_full(R2, blocks["vvvo"], blocks["oovo"]) + W_full(t2, dblocks["vvvo"], dblocks["oovo"])
    D = denominators(inp.eps_o, inp.eps_v)
    R3t = contravariant(WR / (w - D))
    tt = contravariant(W_full(t2, blocks["vvvo"], blocks["oovo"]) / (-D))
    o1a, ota = contractions(R3t, blocks)
    hb = dict(dblocks)
    hb["ovov"] = np.zeros_like(blocks["ovov"])
    o1b, otb = contractions(tt, hb)
    return dict(rho1=o1a + o1b, rho2=back_transform(ota + otb))


def P6(B):
    """The permutation operator P^{abc}_{ijk} of eq. "permutation" (six terms)."""
    return (B + E("jikbac->ijkabc", B) + E("kjicba->ijkabc", B)
            + E("ikjacb->ijkabc", B) + E("jkibca->ijkabc", B)
            + E("kijcab->ijkabc", B))


def L3_full(L1, Lt2, blocks, eps_o, eps_v, w):
    """Covariant L3 of a left state over every ordered i,j,k:
    X^{abc}_{ijk} = L^a_i g_{jbkc} + Lt^{ab}_{ij} F_kc + sum_d Lt^{ad}_{ij} g_{dbkc}
    - sum_l Lt^{ab}_{il} g_{jlkc} (the transposed contractions of Algorithm 1),
    L3 = P X / (w - eps)."""
    X = (E("ia,jbkc->ijkabc", L1, blocks["ovov"]) + E("ijab,kc->ijkabc", Lt2, blocks["F_ov"])
         + E("ijad,dbkc->ijkabc", Lt2, blocks["vvov"])
         - E("ilab,jlkc->ijkabc", Lt2, blocks["ooov"]))
    return P6(X) / (w - denominators(eps_o, eps_v))


def density_full(eps_o, eps_v, t2, blocks, w, L1, L2):
    """Triples contributions of Algorithm 3 by their plain full-tensor sums:
      Dvv_cd =  1/2 sum_{ijkab} L~^{abc}_{ijk} tau^{abd}_{ijk}
      Doo_lk = -1/2 sum_{ijabc} L~^{abc}_{ijk} tau^{abc}_{ijl}
      Dov_kc =  sum_{ijab} Lt^{ab}_{ij} tau~^{abc}_{ijk} - sum_{cik} Y_clik t^{cd}_{ki}
                (the second term at [l][d]), Y_clik = sum_{jab} L~^{abc}_{ijk} t^{ab}_{lj}
    with tau = W / (0 - eps), Lt = the back-transformed L2.  Returns
    dict(Doo, Dov, Dvv, Y, tau, L3)."""
    Lt2 = back_transform(L2)
    tau = W_full(t2, blocks["vvvo"], blocks["oovo"]) / (0.0 - denominators(eps_o, eps_v))
    L3 = L3_full(L1, Lt2, blocks, eps_o, eps_v, w)
    Lc, tc = contravariant(L3), contravariant(tau)
    Y = E("ijkabc,ljab->clik", Lc, t2)
    Dvv = 0.5 * E("ijkabc,ijkabd->cd", Lc, tau)
    Doo = -0.5 * E("ijkabc,ijlabc->lk", Lc, tau)
    Dov = E("ijab,ijkabc->kc", Lt2, tc) - E("clik,kicd->ld", Y, t2)
    return dict(Doo=Doo, Dov=Dov, Dvv=Dvv, Y=Y, tau=tau, L3=L3)
