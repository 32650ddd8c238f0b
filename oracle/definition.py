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
