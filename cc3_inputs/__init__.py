"""Seeded synthetic inputs for the closed-shell CC3 triples hot path.

This module is the only code shared by the FP64 oracle (``oracle/``) and the
GPU library (``paper_2007_01088_gb300``).  It draws random numbers and builds
the input tensors of the problem statement (orbital energies, two-electron
integral blocks, doubles amplitudes in MP2 form, trial vectors); it holds none
of the triples method's arithmetic.

Recipe (the paper's molecules and integrals are not available, so these stand
in for them with the same shapes and value ranges):

* ``eps_o`` ~ U[-1.5, -0.3] Eh, sorted ascending; ``eps_v`` ~ U[0.1, 3.0] Eh,
  sorted ascending.  Optionally the ``n_degenerate`` lowest virtual energies are
  replaced by ``eps_v[0] + U[0, 1e-3]`` (a near-degenerate virtual cluster).
* Cholesky-like vectors ``L[J][p][q] ~ N(0, 0.05^2) * exp(-|p-q|/20)`` drawn for
  ``p <= q`` and mirrored, orbitals ordered occupied first, ``naux`` defaults
  to ``3 * (no + nv)``.  Integrals ``(pq|rs) = sum_J L[J][p][q] L[J][r][s]`` then
  have the full 8-fold permutational symmetry of real orbitals.
* ``F_ov ~ N(0, 1e-3^2)``.
* ``t2[i][j][a][b] = (ai|bj) / (eps_i + eps_j - eps_a - eps_b)`` (MP2 form).
* Frozen core: ``nfrozen`` lowest occupied orbitals are drawn and then dropped;
  every returned tensor covers the active occupied orbitals only.

Array layouts (row-major float64, index order as written):
``t2[i][j][a][b]``, ``g_vvvo[b][d][c][k] = (bd|ck)``,
``g_ooov[l][j][k][c] = (lj|kc)``, ``g_ovov[j][b][k][c] = (jb|kc)``,
``F_ov[k][c]``, ``chol_L[J][p][q]`` over the active orbitals (occupied first).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = ["CC3Inputs", "make_inputs", "make_trial_vectors", "CONFIGS",
           "config_inputs", "unique_triples"]


@dataclass
class CC3Inputs:
    no: int
    nv: int
    eps_o: np.ndarray
    eps_v: np.ndarray
    t2: np.ndarray
    g_vvvo: np.ndarray
    g_ooov: np.ndarray
    g_ovov: np.ndarray
    F_ov: np.ndarray
    chol_L: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def naux(self) -> int:
        return 0 if self.chol_L is None else int(self.chol_L.shape[0])


def _cholesky_vectors(rng, naux: int, n: int) -> np.ndarray:
    raw = rng.normal(0.0, 0.05, size=(naux, n, n))
    p = np.arange(n)
    decay = np.exp(-np.abs(p[:, None] - p[None, :]) / 20.0)
    upper = np.triu(raw * decay)
    return upper + np.transpose(np.triu(upper, 1), (0, 2, 1))


def _block(L: np.ndarray, p: slice, q: slice, r: slice, s: slice) -> np.ndarray:
    """(pq|rs) for orbital ranges p,q,r,s as a dense 4-index array."""
    A = L[:, p, q]
    B = L[:, r, s]
    na, nb = A.shape[1] * A.shape[2], B.shape[1] * B.shape[2]
    out = A.reshape(A.shape[0], na).T @ B.reshape(B.shape[0], nb)
    return out.reshape(A.shape[1], A.shape[2], B.shape[1], B.shape[2])


def make_inputs(no: int, nv: int, seed: int = 0, naux: int | None = None,
                nfrozen: int = 0, n_degenerate: int = 0,
                keep_chol: bool = True) -> CC3Inputs:
    """Draw one seeded synthetic problem with ``no`` active occupied and ``nv``
    virtual orbitals (see the module docstring for the recipe)."""
    if no < 0 or nv < 1:
        raise ValueError("need no >= 0 and nv >= 1")
    rng = np.random.default_rng(seed)
    no_all = no + nfrozen
    n_all = no_all + nv
    if naux is None:
        naux = 3 * (no + nv)
    eps_o_all = np.sort(rng.uniform(-1.5, -0.3, size=no_all))
    eps_v = np.sort(rng.uniform(0.1, 3.0, size=nv))
    if n_degenerate:
        k = min(n_degenerate, nv)
        eps_v[:k] = eps_v[0] + rng.uniform(0.0, 1e-3, size=k)
        eps_v = np.sort(eps_v)
    L_all = _cholesky_vectors(rng, naux, n_all)
    F_ov = rng.normal(0.0, 1e-3, size=(no, nv))

    act = np.r_[nfrozen:no_all, no_all:n_all]
    L = np.ascontiguousarray(L_all[:, act][:, :, act])
    o = slice(0, no)
    v = slice(no, no + nv)
    g_vvvo = _block(L, v, v, v, o)
    g_ooov = _block(L, o, o, o, v)
    g_ovov = _block(L, o, v, o, v)
    eps_o = eps_o_all[nfrozen:]
    # (ai|bj) = (ia|jb) = g_ovov[i][a][j][b]; t2[i][j][a][b] in MP2 form
    D = (eps_o[:, None, None, None] + eps_o[None, :, None, None]
         - eps_v[None, None, :, None] - eps_v[None, None, None, :])
    t2 = np.transpose(g_ovov, (0, 2, 1, 3)) / D
    meta = dict(seed=seed, naux=naux, nfrozen=nfrozen,
                n_degenerate=n_degenerate)
    return CC3Inputs(no=no, nv=nv, eps_o=np.ascontiguousarray(eps_o),
                     eps_v=eps_v, t2=np.ascontiguousarray(t2),
                     g_vvvo=np.ascontiguousarray(g_vvvo),
                     g_ooov=np.ascontiguousarray(g_ooov),
                     g_ovov=np.ascontiguousarray(g_ovov),
                     F_ov=np.ascontiguousarray(F_ov),
                     chol_L=L if keep_chol else None, meta=meta)


def make_trial_vectors(no: int, nv: int, nvec: int, seed: int = 1):
    """Seeded trial vectors: R1 ~ N(0, 0.1^2), R2 ~ N(0, 0.01^2) made pair
    symmetric (R2[i,j,a,b] = R2[j,i,b,a]) and each (R1, R2) normalised to unit
    Euclidean norm.  Returns R1[nvec][no][nv], R2[nvec][no][no][nv][nv]."""
    rng = np.random.default_rng(seed)
    R1 = np.empty((nvec, no, nv))
    R2 = np.empty((nvec, no, no, nv, nv))
    for n in range(nvec):
        r1 = rng.normal(0.0, 0.1, size=(no, nv))
        x = rng.normal(0.0, 0.01, size=(no, no, nv, nv))
        r2 = 0.5 * (x + np.transpose(x, (1, 0, 3, 2)))
        nrm = math.sqrt(float(np.sum(r1 * r1) + np.sum(r2 * r2)))
        if nrm == 0.0:
            nrm = 1.0
        R1[n] = r1 / nrm
        R2[n] = r2 / nrm
    return R1, R2


def unique_triples(no: int):
    """The occupied triples i >= j >= k with not all three equal, in loop
    order (i outermost), each with its number of distinct permutations."""
    out = []
    for i in range(no):
        for j in range(i + 1):
            for k in range(j + 1):
                if i == j == k:
                    continue
                w = 6 if (i != j and j != k) else 3
                out.append((i, j, k, w))
    return out


# The five workloads the hot path is measured and tested on.
CONFIGS = {
    "cfg1_no5_nv30": dict(no=5, nv=30, seed=0),
    "cfg2_no16_nv160": dict(no=16, nv=160, seed=0),
    "cfg3_proline_no22_nv250": dict(no=22, nv=250, seed=0, naux=700, nfrozen=9,
                                    n_degenerate=10),
    "cfg4_jacobian_no20_nv200": dict(no=20, nv=200, seed=0),
}


def config_inputs(name: str, **over) -> CC3Inputs:
    kw = dict(CONFIGS[name])
    kw.update(over)
    return make_inputs(**kw)
