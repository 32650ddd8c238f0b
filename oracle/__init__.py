"""FP64 CPU oracle for the CC3 triples hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package never imports the product library: the two share nothing but the
seeded input generator in ``cc3_inputs``.

Two independent forms of the same result (Paul, Myhre, Koch, arXiv 2007.01088):

* ``omega`` / ``prep`` / ``jacobian`` / ``left_jacobian`` / ``density``: the
  restricted-loop algorithms written out in plain C (``cc3_oracle.c``;
  Algorithm 1, Algorithm 2, the right Jacobian transformation reconstructed
  from eq. "jcc3", its transpose, and Algorithm 3's densities).
* ``matrix_form``: the same restricted loops with numpy matrix products as
  steps, for test shapes where the C loops are too slow.
* ``definition.omega_full`` / ``definition.density_full``: the plain
  definitions over the full nv^3 no^3 tensor (every ordered i,j,k), numpy,
  tiny sizes only.

``t1_transform`` gives T1-transformed integral blocks, used to pin the Jacobian
as the derivative of the residual (finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O3 -fopenmp, portable flags)."""
    src = os.path.join(_HERE, "cc3_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.oracle_omega.argtypes = [I, I] + [P] * 9 + [I, P, P, P, P, P, P, I]
            lib.oracle_omega.restype = I
            lib.oracle_prep.argtypes = [I, I] + [P] * 6 + [I, P, P, P, P, I]
            lib.oracle_prep.restype = I
            lib.oracle_jacobian.argtypes = ([I, I] + [P] * 9 + [P, I, I, P, P, P]
                                            + [I, P, P, P, P, I])
            lib.oracle_jacobian.restype = I
            lib.oracle_left_jacobian.argtypes = ([I, I] + [P] * 9 + [P, I, I, P, P, P]
                                                 + [I, P, P, P, P, I])
            lib.oracle_left_jacobian.restype = I
            lib.oracle_density.argtypes = ([I, I] + [P] * 9 + [ctypes.c_double, P, P]
                                           + [P, P, P, P, I])
            lib.oracle_density.restype = I
            lib.oracle_dressed_blocks.argtypes = [I, I, P, I, P, P, P, P, P, P]
            lib.oracle_dressed_blocks.restype = None
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def symmetric_blocks(inp):
    """The general five blocks from the symmetric (T1 = 0) inputs:
    vvvo g_bdck, oovo g_ljck = (lj|kc), ooov g_jlkc, ovov g_jbkc,
    vvov g_dbkc = (bd|ck)."""
    vvvo = _c(inp.g_vvvo)
    oovo = _c(np.transpose(inp.g_ooov, (0, 1, 3, 2)))
    ooov = _c(inp.g_ooov)
    ovov = _c(inp.g_ovov)
    vvov = _c(np.transpose(inp.g_vvvo, (1, 0, 3, 2)))
    return dict(vvvo=vvvo, oovo=oovo, ooov=ooov, ovov=ovov, vvov=vvov,
                F_ov=_c(inp.F_ov))


def _triples_arg(triples):
    if triples is None:
        return 0, None
    arr = np.ascontiguousarray(np.asarray(triples, dtype=np.int32).reshape(-1, 3))
    return int(arr.shape[0]), arr


def omega(no, nv, eps_o, eps_v, t2, blocks, triples=None, nthreads=0):
    """Algorithm 1 on the general blocks.  Returns dict(omega1, omega2,
    omega2_tilde, E_T, flops, threads)."""
    lib = _load()
    eps_o, eps_v, t2 = _c(eps_o), _c(eps_v), _c(t2)
    b = {k: _c(v) for k, v in blocks.items()}
    om1 = np.zeros((no, nv))
    om2 = np.zeros((no, no, nv, nv))
    omt = np.zeros((no, no, nv, nv))
    et = ctypes.c_double(0.0)
    fl = ctypes.c_longlong(0)
    nt, tri = _triples_arg(triples)
    used = lib.oracle_omega(no, nv, _p(eps_o), _p(eps_v), _p(t2), _p(b["vvvo"]),
                            _p(b["oovo"]), _p(b["ooov"]), _p(b["ovov"]),
                            _p(b["vvov"]), _p(b["F_ov"]), nt, _p(tri), _p(om1),
                            _p(om2), _p(omt), ctypes.byref(et), ctypes.byref(fl),
                            int(nthreads))
    if used < 0:
        raise MemoryError("oracle_omega failed")
    return dict(omega1=om1, omega2=om2, omega2_tilde=omt, E_T=et.value,
                flops=fl.value, threads=used)


def omega_inputs(inp, triples=None, nthreads=0):
    """Algorithm 1 on a ``cc3_inputs.CC3Inputs`` problem."""
    return omega(inp.no, inp.nv, inp.eps_o, inp.eps_v, inp.t2,
                 symmetric_blocks(inp), triples, nthreads)


def prep(inp, triples=None, nthreads=0):
    """Algorithm 2 intermediates Zv[a][b][i][d], Zo[a][j][i][l]."""
    lib = _load()
    no, nv = inp.no, inp.nv
    b = symmetric_blocks(inp)
    Zv = np.zeros((nv, nv, no, nv))
    Zo = np.zeros((nv, no, no, no))
    fl = ctypes.c_longlong(0)
    nt, tri = _triples_arg(triples)
    used = lib.oracle_prep(no, nv, _p(_c(inp.eps_o)), _p(_c(inp.eps_v)),
                           _p(_c(inp.t2)), _p(b["vvvo"]), _p(b["oovo"]),
                           _p(b["ovov"]), nt, _p(tri), _p(Zv), _p(Zo),
                           ctypes.byref(fl), int(nthreads))
    if used < 0:
        raise MemoryError("oracle_prep failed")
    return dict(Zv=Zv, Zo=Zo, flops=fl.value, threads=used)


def jacobian(inp, R1, R2, w, triples=None, nthreads=0):
    """Right Jacobian transformation of trial vectors R1[n][i][a],
    R2[n][i][j][a][b] at frequencies w[n].  Returns dict(rho1, rho2, flops)."""
    lib = _load()
    no, nv = inp.no, inp.nv
    if inp.chol_L is None:
        raise ValueError("the Jacobian needs the Cholesky vectors")
    b = symmetric_blocks(inp)
    R1 = _c(R1).reshape(-1, no, nv)
    nvec = R1.shape[0]
    R2 = _c(R2).reshape(nvec, no, no, nv, nv)
    w = _c(np.broadcast_to(np.asarray(w, dtype=np.float64), (nvec,)))
    L = _c(inp.chol_L)
    rho1 = np.zeros((nvec, no, nv))
    rho2 = np.zeros((nvec, no, no, nv, nv))
    fl = ctypes.c_longlong(0)
    nt, tri = _triples_arg(triples)
    used = lib.oracle_jacobian(no, nv, _p(_c(inp.eps_o)), _p(_c(inp.eps_v)),
                               _p(_c(inp.t2)), _p(b["vvvo"]), _p(b["oovo"]),
                               _p(b["ooov"]), _p(b["ovov"]), _p(b["vvov"]),
                               _p(b["F_ov"]), _p(L), int(L.shape[0]), nvec,
                               _p(w), _p(R1), _p(R2), nt, _p(tri), _p(rho1),
                               _p(rho2), ctypes.byref(fl), int(nthreads))
    if used < 0:
        raise MemoryError("oracle_jacobian failed")
    return dict(rho1=rho1, rho2=rho2, flops=fl.value, threads=used)


def left_jacobian(inp, L1, L2, w, triples=None, nthreads=0):
    """Left (transpose) Jacobian transformation of left vectors L1[n][i][a],
    L2[n][i][j][a][b] at frequencies w[n]: the exact transpose of
    ``jacobian`` under the plain inner product over (R1, R2) elements
    (sigma2 projected on pair-symmetric tensors).  Returns dict(sigma1,
    sigma2, flops)."""
    lib = _load()
    no, nv = inp.no, inp.nv
    if inp.chol_L is None:
        raise ValueError("the Jacobian needs the Cholesky vectors")
    b = symmetric_blocks(inp)
    L1 = _c(L1).reshape(-1, no, nv)
    nvec = L1.shape[0]
    L2 = _c(L2).reshape(nvec, no, no, nv, nv)
    w = _c(np.broadcast_to(np.asarray(w, dtype=np.float64), (nvec,)))
    L = _c(inp.chol_L)
    s1 = np.zeros((nvec, no, nv))
    s2 = np.zeros((nvec, no, no, nv, nv))
    fl = ctypes.c_longlong(0)
    nt, tri = _triples_arg(triples)
    used = lib.oracle_left_jacobian(no, nv, _p(_c(inp.eps_o)), _p(_c(inp.eps_v)),
                                    _p(_c(inp.t2)), _p(b["vvvo"]), _p(b["oovo"]),
                                    _p(b["ooov"]), _p(b["ovov"]), _p(b["vvov"]),
                                    _p(b["F_ov"]), _p(L), int(L.shape[0]), nvec,
                                    _p(w), _p(L1), _p(L2), nt, _p(tri), _p(s1),
                                    _p(s2), ctypes.byref(fl), int(nthreads))
    if used < 0:
        raise MemoryError("oracle_left_jacobian failed")
    return dict(sigma1=s1, sigma2=s2, flops=fl.value, threads=used)


def density(no, nv, eps_o, eps_v, t2, blocks, w, L1, L2, nthreads=0):
    """Algorithm 3 on the general blocks: the triples contributions to the
    one-electron density D^{m,0} of the left state (L1[i][a], L2[i][j][a][b])
    at frequency w (w = 0 with ground-state multipliers: D^{0,0}).  Returns
    dict(Doo[no][no], Dov[no][nv], Dvv[nv][nv], flops, threads); the vo block
    has no triples term."""
    lib = _load()
    b = {k: _c(v) for k, v in blocks.items()}
    L1, L2 = _c(L1).reshape(no, nv), _c(L2).reshape(no, no, nv, nv)
    doo, dov, dvv = np.zeros((no, no)), np.zeros((no, nv)), np.zeros((nv, nv))
    fl = ctypes.c_longlong(0)
    used = lib.oracle_density(no, nv, _p(_c(eps_o)), _p(_c(eps_v)), _p(_c(t2)),
                              _p(b["vvvo"]), _p(b["oovo"]), _p(b["ooov"]), _p(b["ovov"]),
                              _p(b["vvov"]), _p(b["F_ov"]), float(w), _p(L1), _p(L2),
                              _p(doo), _p(dov), _p(dvv), ctypes.byref(fl), int(nthreads))
    if used < 0:
        raise MemoryError("oracle_density failed")
    return dict(Doo=doo, Dov=dov, Dvv=dvv, flops=fl.value, threads=used)


def density_inputs(inp, w, L1, L2, nthreads=0):
    """``density`` on the symmetric (T1 = 0) inputs of ``cc3_inputs``."""
    return density(inp.no, inp.nv, inp.eps_o, inp.eps_v, inp.t2, symmetric_blocks(inp),
                   w, L1, L2, nthreads)


def dressed_blocks(inp, R1):
    """The R1-dressed blocks (vvvo, oovo, ooov, vvov, F) of the Jacobian."""
    lib = _load()
    no, nv = inp.no, inp.nv
    L = _c(inp.chol_L)
    out = dict(vvvo=np.zeros((nv, nv, nv, no)), oovo=np.zeros((no, no, nv, no)),
               ooov=np.zeros((no, no, no, nv)), vvov=np.zeros((nv, nv, no, nv)),
               F_ov=np.zeros((no, nv)))
    lib.oracle_dressed_blocks(no, nv, _p(L), int(L.shape[0]), _p(_c(R1)),
                              _p(out["vvvo"]), _p(out["oovo"]), _p(out["ooov"]),
                              _p(out["vvov"]), _p(out["F_ov"]))
    return out


def t1_transform(inp, t1):
    return {k: _c(x) for k, x in t1_transform_complex(inp, t1).items()}


def t1_transform_complex(inp, t1):
    """Integral blocks and F_ov in the T1-transformed basis of
    H = exp(-T1) H exp(T1) (t1[i][a] = t^a_i): every Cholesky vector becomes
    X L^J Y^T with X = 1 - t1 (virtual rows) and Y = 1 + t1^T (occupied rows),
    so g~_pqrs = sum_J L~^J_pq L~^J_rs.  F~_kc = F_kc + sum_l [2 (g~ - g)_kcll
    - (g~ - g)_kllc] (h_kc is unchanged by the transformation).  Returns the
    general five blocks of the residual."""
    no, nv = inp.no, inp.nv
    n = no + nv
    L = inp.chol_L
    t1 = np.asarray(t1)
    t1m = np.zeros((n, n), dtype=np.result_type(t1.dtype, np.float64))
    t1m[no:, :no] = t1.T          # t1m[a][i] = t^a_i
    X = np.eye(n) - t1m
    Y = np.eye(n) + t1m.T
    Lt = np.einsum("pt,Jtu,qu->Jpq", X, L, Y, optimize=True)
    o, v = slice(0, no), slice(no, n)

    def blk(Lx, p, q, r, s):
        return np.einsum("Jpq,Jrs->pqrs", Lx[:, p, q], Lx[:, r, s], optimize=True)

    out = dict(vvvo=blk(Lt, v, v, v, o), oovo=blk(Lt, o, o, v, o),
               ooov=blk(Lt, o, o, o, v), ovov=blk(Lt, o, v, o, v),
               vvov=blk(Lt, v, v, o, v))
    dJ = (np.einsum("Jkc,Jll->kc", Lt[:, o, v], Lt[:, o, o])
          - np.einsum("Jkc,Jll->kc", L[:, o, v], L[:, o, o]))
    dK = (np.einsum("Jkl,Jlc->kc", Lt[:, o, o], Lt[:, o, v])
          - np.einsum("Jkl,Jlc->kc", L[:, o, o], L[:, o, v]))
    out["F_ov"] = np.asarray(inp.F_ov) + 2.0 * dJ - dK
    return {k: np.ascontiguousarray(x) for k, x in out.items()}


from . import definition  # noqa: E402  (numpy full-tensor definition)
