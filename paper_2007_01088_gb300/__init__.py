"""GB300 (sm_103a) CC3 triples library: Python binding of libcc3.so.

The functions here carry the names of the C ABI in ``include/cc3.h`` and only
marshal arguments; every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: if the shared library cannot be loaded,
importing the binding raises.

Arrays may be numpy float64 arrays (host; the library copies and synchronises)
or CUDA torch float64 tensors (device; the context is then created with
CC3_DEVICE_PTRS and every call takes device tensors).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB, build as _build

__all__ = ["CC3_FP64", "CC3_SPLIT_BF16", "CC3_SPLIT_INT8", "CC3_DEVICE_PTRS",
           "CC3_DETERMINISTIC", "CC3Error", "lib", "cc3_ctx_create",
           "cc3_ctx_destroy", "cc3_ctx_set_triples", "cc3_omega_triples",
           "cc3_jacobian_triples", "cc3_ctx_counters", "cc3_ctx_set_slices",
           "cc3_strerror", "cc3_cvs_triples", "cc3_denominator_gap", "CC3_DENOM_MIN",
           "cc3_left_jacobian_triples", "cc3_density_triples", "Context", "EXPORTED"]

CC3_FP64, CC3_SPLIT_BF16, CC3_SPLIT_INT8 = 0, 1, 2
CC3_DEVICE_PTRS, CC3_DETERMINISTIC = 1, 2
CC3_DENOM_MIN = 1e-6  # Eh, smallest |w - eps| the Jacobian accepts
(CC3_OK, CC3_ERR_ARG, CC3_ERR_OOM, CC3_ERR_CUDA, CC3_ERR_TIMEOUT, CC3_ERR_DENOM, CC3_ERR_BUSY,
 CC3_ERR_UNSUPPORTED, CC3_ERR_NOT_FOUND, CC3_ERR_CANCELLED) = range(0, -10, -1)

# every symbol include/cc3.h declares
EXPORTED = ["cc3_ctx_create", "cc3_ctx_destroy", "cc3_ctx_set_triples",
            "cc3_omega_triples", "cc3_jacobian_triples", "cc3_ctx_counters",
            "cc3_ctx_set_slices", "cc3_strerror", "cc3_serve_start",
            "cc3_serve_submit", "cc3_serve_poll", "cc3_serve_wait",
            "cc3_serve_cancel", "cc3_serve_stats", "cc3_serve_stop",
            "cc3_debug_split_gemm", "cc3_last_error", "cc3_ctx_set_tracing",
            "cc3_ctx_trace", "cc3_omega_triples_noalloc", "cc3_serve_footprint",
            "cc3_ctx_autotune", "cc3_ctx_get_tuning", "cc3_cvs_triples",
            "cc3_denominator_gap", "cc3_debug_wait_timeout", "cc3_ctx_create_general",
            "cc3_left_jacobian_triples", "cc3_density_triples"]


class CC3Error(RuntimeError):
    def __init__(self, status: int, where: str):
        detail = lib.cc3_last_error().decode()
        super().__init__(f"{where}: {cc3_strerror(status)} ({status}) [{detail}]")
        self.status = status


class TraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong),
                ("ms", ctypes.c_double), ("flop", ctypes.c_double),
                ("slice_flop", ctypes.c_double)]


class Trace(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("e", TraceEntry * 8)]


class Counters(ctypes.Structure):
    _fields_ = [("nominal_flop", ctypes.c_double), ("executed_flop", ctypes.c_double),
                ("launches", ctypes.c_longlong), ("slices", ctypes.c_int)]


class Request(ctypes.Structure):
    """cc3_request: one residual (kind 0) or Jacobian (kind 1) evaluation."""
    _fields_ = ([("kind", ctypes.c_int), ("prec", ctypes.c_int), ("no", ctypes.c_int),
                 ("nv", ctypes.c_int), ("naux", ctypes.c_int)]
                + [(n, ctypes.c_void_p) for n in ("eps_o", "eps_v", "t2", "g_vvvo", "g_ooov",
                                                  "g_ovov", "F_ov", "chol_L")]
                + [("nvec", ctypes.c_int)]
                + [(n, ctypes.c_void_p) for n in ("omega", "R1", "R2", "Omega1", "Omega2",
                                                  "E_T", "rho1", "rho2")]
                + [("flags", ctypes.c_uint)])


class Stats(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_longlong) for n in ("submitted", "admitted", "completed",
                                                  "rejected", "cancelled")]
                + [(n, ctypes.c_double) for n in ("p50_ms", "p99_ms", "mean_ms", "busy_s",
                                                  "wall_s", "nominal_flop")]
                + [("hbm_in_use", ctypes.c_size_t), ("hbm_peak", ctypes.c_size_t)])


def _load():
    path = LIB
    if not os.path.exists(path):
        path = _build()
    L = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.cc3_ctx_create.argtypes = [ctypes.POINTER(P), I, I] + [P] * 8 + [I, ctypes.c_uint, P]
    L.cc3_ctx_create.restype = I
    L.cc3_ctx_create_general.argtypes = [ctypes.POINTER(P), I, I] + [P] * 9 + [ctypes.c_uint, P]
    L.cc3_ctx_create_general.restype = I
    L.cc3_ctx_destroy.argtypes = [P]
    L.cc3_ctx_destroy.restype = None
    L.cc3_ctx_set_triples.argtypes = [P, I, P]
    L.cc3_ctx_set_triples.restype = I
    L.cc3_cvs_triples.argtypes = [I, I, P, I, P]
    L.cc3_cvs_triples.restype = I
    L.cc3_denominator_gap.argtypes = [I, I, P, P, I, P, D, ctypes.POINTER(D)]
    L.cc3_denominator_gap.restype = I
    L.cc3_omega_triples.argtypes = [P, I, P, P, P, P]
    L.cc3_omega_triples.restype = I
    L.cc3_jacobian_triples.argtypes = [P, I, I, P, P, P, P, P, P]
    L.cc3_jacobian_triples.restype = I
    L.cc3_left_jacobian_triples.argtypes = [P, I, I, P, P, P, P, P, P]
    L.cc3_left_jacobian_triples.restype = I
    L.cc3_density_triples.argtypes = [P, I, ctypes.c_double, P, P, P, P, P, P]
    L.cc3_density_triples.restype = I
    L.cc3_ctx_counters.argtypes = [P, ctypes.POINTER(Counters)]
    L.cc3_ctx_counters.restype = I
    L.cc3_ctx_set_slices.argtypes = [P, I]
    L.cc3_ctx_set_slices.restype = I
    L.cc3_debug_split_gemm.argtypes = [I, I, I, P, P, P, I]
    L.cc3_debug_split_gemm.restype = I
    L.cc3_debug_wait_timeout.argtypes = [D]
    L.cc3_debug_wait_timeout.restype = I
    L.cc3_ctx_set_tracing.argtypes = [P, I]
    L.cc3_ctx_set_tracing.restype = I
    L.cc3_ctx_trace.argtypes = [P, ctypes.POINTER(Trace)]
    L.cc3_ctx_trace.restype = I
    L.cc3_omega_triples_noalloc.argtypes = [I, I] + [P] * 7 + [P, P, P, P]
    L.cc3_omega_triples_noalloc.restype = I
    IP = ctypes.POINTER(I)
    L.cc3_ctx_autotune.argtypes = [P, P, IP, IP]
    L.cc3_ctx_autotune.restype = I
    L.cc3_ctx_get_tuning.argtypes = [P, IP, IP]
    L.cc3_ctx_get_tuning.restype = I
    RP = ctypes.POINTER(Request)
    L.cc3_serve_start.argtypes = [ctypes.POINTER(P), ctypes.c_size_t, I]
    L.cc3_serve_start.restype = I
    L.cc3_serve_footprint.argtypes = [RP, ctypes.POINTER(ctypes.c_size_t)]
    L.cc3_serve_footprint.restype = I
    L.cc3_serve_submit.argtypes = [P, RP, ctypes.POINTER(ctypes.c_uint64)]
    L.cc3_serve_submit.restype = I
    L.cc3_serve_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(I)]
    L.cc3_serve_poll.restype = I
    L.cc3_serve_wait.argtypes = [P, ctypes.c_uint64, D]
    L.cc3_serve_wait.restype = I
    L.cc3_serve_cancel.argtypes = [P, ctypes.c_uint64]
    L.cc3_serve_cancel.restype = I
    L.cc3_serve_stats.argtypes = [P, ctypes.POINTER(Stats)]
    L.cc3_serve_stats.restype = I
    L.cc3_serve_stop.argtypes = [P]
    L.cc3_serve_stop.restype = I
    L.cc3_last_error.argtypes = []
    L.cc3_last_error.restype = ctypes.c_char_p
    L.cc3_strerror.argtypes = [I]
    L.cc3_strerror.restype = ctypes.c_char_p
    return L


lib = _load()


def cc3_last_error() -> str:
    return lib.cc3_last_error().decode()


def cc3_strerror(status: int) -> str:
    return lib.cc3_strerror(int(status)).decode()


def _check(status, where):
    if status != 0:
        raise CC3Error(status, where)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """Pointer of a numpy array or torch tensor (None for None)."""
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if not (isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]):
        raise ValueError("arrays must be C-contiguous")
    return x.ctypes.data_as(ctypes.c_void_p)


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


# ---- C ABI, same names -----------------------------------------------------
def cc3_ctx_create(no, nv, eps_o, eps_v, t2, g_vvvo, g_ooov, g_ovov, F_ov,
                   chol_L=None, naux=0, flags=0, stream=None):
    ctx = ctypes.c_void_p()
    st = lib.cc3_ctx_create(ctypes.byref(ctx), int(no), int(nv), _ptr(eps_o),
                            _ptr(eps_v), _ptr(t2), _ptr(g_vvvo), _ptr(g_ooov),
                            _ptr(g_ovov), _ptr(F_ov), _ptr(chol_L), int(naux),
                            int(flags), _stream(stream))
    _check(st, "cc3_ctx_create")
    return ctx


def cc3_ctx_create_general(no, nv, eps_o, eps_v, t2, g_vvvo, g_oovo, g_ooov, g_ovov, g_vvov,
                           F_ov, flags=0, stream=None):
    ctx = ctypes.c_void_p()
    st = lib.cc3_ctx_create_general(ctypes.byref(ctx), int(no), int(nv), _ptr(eps_o),
                                    _ptr(eps_v), _ptr(t2), _ptr(g_vvvo), _ptr(g_oovo),
                                    _ptr(g_ooov), _ptr(g_ovov), _ptr(g_vvov), _ptr(F_ov),
                                    int(flags), _stream(stream))
    _check(st, "cc3_ctx_create_general")
    return ctx


def cc3_ctx_destroy(ctx):
    lib.cc3_ctx_destroy(ctx)


def cc3_ctx_set_triples(ctx, triples=None):
    if triples is None or len(triples) == 0:
        _check(lib.cc3_ctx_set_triples(ctx, 0, None), "cc3_ctx_set_triples")
        return
    arr = np.ascontiguousarray(np.asarray(triples, dtype=np.int32).reshape(-1, 3))
    _check(lib.cc3_ctx_set_triples(ctx, int(arr.shape[0]), arr.ctypes.data_as(ctypes.c_void_p)),
           "cc3_ctx_set_triples")


def cc3_cvs_triples(no, core):
    """The occupied triples i >= j >= k (not all equal) with at least one index
    in `core` (core-valence separation), as an (n, 3) int32 array."""
    c = np.ascontiguousarray(np.asarray(core, dtype=np.int32).reshape(-1))
    cp = c.ctypes.data_as(ctypes.c_void_p) if c.size else None
    n = lib.cc3_cvs_triples(int(no), int(c.size), cp, 0, None)
    if n < 0:
        _check(n, "cc3_cvs_triples")
    out = np.zeros((max(n, 1), 3), dtype=np.int32)
    m = lib.cc3_cvs_triples(int(no), int(c.size), cp, int(n), out.ctypes.data_as(ctypes.c_void_p))
    if m < 0:
        _check(m, "cc3_cvs_triples")
    return out[:n]


def cc3_denominator_gap(no, nv, eps_o, eps_v, w, triples=None):
    """Smallest |w - eps^{abc}_{ijk}| over every virtual triple and the occupied
    triples of the loop (all i >= j >= k, not all equal, when triples is None).
    Host only."""
    eo = np.ascontiguousarray(eps_o, dtype=np.float64)
    ev = np.ascontiguousarray(eps_v, dtype=np.float64)
    if triples is None or len(triples) == 0:
        n, tp = 0, None
    else:
        arr = np.ascontiguousarray(np.asarray(triples, dtype=np.int32).reshape(-1, 3))
        n, tp = int(arr.shape[0]), arr.ctypes.data_as(ctypes.c_void_p)
    gap = ctypes.c_double(0.0)
    _check(lib.cc3_denominator_gap(int(no), int(nv), _ptr(eo), _ptr(ev), n, tp, float(w),
                                   ctypes.byref(gap)), "cc3_denominator_gap")
    return gap.value


def cc3_omega_triples(ctx, prec, Omega1, Omega2, E_T, stream=None):
    _check(lib.cc3_omega_triples(ctx, int(prec), _ptr(Omega1), _ptr(Omega2), _ptr(E_T),
                                 _stream(stream)), "cc3_omega_triples")


def cc3_jacobian_triples(ctx, prec, nvec, omega, R1, R2, rho1, rho2, stream=None):
    w = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).reshape(-1))
    _check(lib.cc3_jacobian_triples(ctx, int(prec), int(nvec), w.ctypes.data_as(ctypes.c_void_p),
                                    _ptr(R1), _ptr(R2), _ptr(rho1), _ptr(rho2),
                                    _stream(stream)), "cc3_jacobian_triples")


def cc3_left_jacobian_triples(ctx, prec, nvec, omega, L1, L2, sigma1, sigma2, stream=None):
    w = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).reshape(-1))
    _check(lib.cc3_left_jacobian_triples(ctx, int(prec), int(nvec),
                                         w.ctypes.data_as(ctypes.c_void_p), _ptr(L1), _ptr(L2),
                                         _ptr(sigma1), _ptr(sigma2), _stream(stream)),
           "cc3_left_jacobian_triples")


def cc3_density_triples(ctx, prec, omega, L1, L2, D_oo, D_ov, D_vv, stream=None):
    _check(lib.cc3_density_triples(ctx, int(prec), float(omega), _ptr(L1), _ptr(L2), _ptr(D_oo),
                                   _ptr(D_ov), _ptr(D_vv), _stream(stream)),
           "cc3_density_triples")


def cc3_ctx_counters(ctx):
    c = Counters()
    _check(lib.cc3_ctx_counters(ctx, ctypes.byref(c)), "cc3_ctx_counters")
    return dict(nominal_flop=c.nominal_flop, executed_flop=c.executed_flop,
                launches=c.launches, slices=c.slices)


def cc3_omega_triples_noalloc(no, nv, eps_o, eps_v, t2, g_vvvo, g_ooov, g_ovov, F_ov,
                              Omega1, Omega2, E_T, stream=None):
    """FP64 residual with no device allocation (all arguments CUDA tensors)."""
    _check(lib.cc3_omega_triples_noalloc(int(no), int(nv), _ptr(eps_o), _ptr(eps_v), _ptr(t2),
                                         _ptr(g_vvvo), _ptr(g_ooov), _ptr(g_ovov), _ptr(F_ov),
                                         _ptr(Omega1), _ptr(Omega2), _ptr(E_T),
                                         _stream(stream)), "cc3_omega_triples_noalloc")


def cc3_ctx_set_tracing(ctx, on=True):
    _check(lib.cc3_ctx_set_tracing(ctx, int(bool(on))), "cc3_ctx_set_tracing")


def cc3_ctx_trace(ctx):
    """Per kernel class of the last call: launches, ms, flop, slice_flop."""
    t = Trace()
    _check(lib.cc3_ctx_trace(ctx, ctypes.byref(t)), "cc3_ctx_trace")
    return {t.e[i].name.decode(): dict(launches=t.e[i].launches, ms=t.e[i].ms,
                                       flop=t.e[i].flop, slice_flop=t.e[i].slice_flop)
            for i in range(t.n)}


def cc3_ctx_autotune(ctx, stream=None):
    """Tunes the split path's tiling; returns (ksteps_per_tile, ntile_w)."""
    ks, nt = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib.cc3_ctx_autotune(ctx, _stream(stream), ctypes.byref(ks), ctypes.byref(nt)),
           "cc3_ctx_autotune")
    return ks.value, nt.value


def cc3_ctx_get_tuning(ctx):
    ks, nt = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib.cc3_ctx_get_tuning(ctx, ctypes.byref(ks), ctypes.byref(nt)), "cc3_ctx_get_tuning")
    return ks.value, nt.value


def cc3_ctx_set_slices(ctx, slices):
    _check(lib.cc3_ctx_set_slices(ctx, int(slices)), "cc3_ctx_set_slices")


def cc3_debug_wait_timeout(limit_s=1e-3):
    """Runs a bounded device wait that cannot succeed; returns its status
    (CC3_ERR_TIMEOUT expected)."""
    return lib.cc3_debug_wait_timeout(float(limit_s))


def cc3_debug_split_gemm(A, B, slices=6):
    """C = A @ B.T through the split-precision tensor-core engine (diagnostic)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[0]
    C = np.zeros((M, N))
    _check(lib.cc3_debug_split_gemm(M, N, K, _ptr(A), _ptr(B), _ptr(C), int(slices)),
           "cc3_debug_split_gemm")
    return C


# ---- convenience wrapper -----------------------------------------------------
class Context:
    """Owns one cc3_ctx.  ``inputs`` has the fields of cc3_inputs.CC3Inputs
    (no, nv, eps_o, eps_v, t2, g_vvvo, g_ooov, g_ovov, F_ov, chol_L).  With
    ``device=True`` the inputs are uploaded through torch CUDA tensors and the
    context works on device pointers."""

    def __init__(self, inputs, device: bool = False, stream=None, flags: int = 0,
                 blocks=None):
        """blocks: the five general (e.g. T1-transformed) integral blocks and
        F_ov as a dict (vvvo, oovo, ooov, ovov, vvov, F_ov); the context is
        then created with cc3_ctx_create_general and inputs supplies the
        sizes, the orbital energies and t2."""
        self.no, self.nv = int(inputs.no), int(inputs.nv)
        self.device = device
        self.stream = stream
        L = getattr(inputs, "chol_L", None) if blocks is None else None
        names = ["eps_o", "eps_v", "t2", "g_vvvo", "g_ooov", "g_ovov", "F_ov"]
        if blocks is None:
            arrs = {n: np.ascontiguousarray(getattr(inputs, n), dtype=np.float64) for n in names}
        else:
            arrs = {n: np.ascontiguousarray(getattr(inputs, n), dtype=np.float64)
                    for n in ("eps_o", "eps_v", "t2")}
            for k in ("vvvo", "oovo", "ooov", "ovov", "vvov"):
                arrs["g_" + k] = np.ascontiguousarray(blocks[k], dtype=np.float64)
            arrs["F_ov"] = np.ascontiguousarray(blocks["F_ov"], dtype=np.float64)
        if L is not None:
            arrs["chol_L"] = np.ascontiguousarray(L, dtype=np.float64)
        if device:
            import torch
            self._keep = {n: torch.from_numpy(a).cuda() for n, a in arrs.items()}
            src = self._keep
            flags |= CC3_DEVICE_PTRS
        else:
            src = arrs
        naux = 0 if L is None else int(L.shape[0])
        if blocks is None:
            self.ctx = cc3_ctx_create(self.no, self.nv, src["eps_o"], src["eps_v"], src["t2"],
                                      src["g_vvvo"], src["g_ooov"], src["g_ovov"], src["F_ov"],
                                      src.get("chol_L"), naux, flags, stream)
        else:
            self.ctx = cc3_ctx_create_general(self.no, self.nv, src["eps_o"], src["eps_v"],
                                              src["t2"], src["g_vvvo"], src["g_oovo"],
                                              src["g_ooov"], src["g_ovov"], src["g_vvov"],
                                              src["F_ov"], flags, stream)
        if device:
            import torch
            torch.cuda.synchronize()
            self._keep = None

    def close(self):
        if getattr(self, "ctx", None):
            cc3_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_triples(self, triples=None):
        cc3_ctx_set_triples(self.ctx, triples)

    def set_cvs(self, core):
        """Restrict the context to the triples that contain a core orbital of
        `core` (core-valence separation); returns those triples."""
        tr = cc3_cvs_triples(self.no, core)
        if len(tr) == 0:
            raise CC3Error(CC3_ERR_ARG, "set_cvs: no triple contains a core index")
        cc3_ctx_set_triples(self.ctx, tr)
        return tr

    def set_slices(self, s):
        cc3_ctx_set_slices(self.ctx, s)

    def autotune(self):
        return cc3_ctx_autotune(self.ctx, self.stream)

    def tuning(self):
        return cc3_ctx_get_tuning(self.ctx)

    def counters(self):
        return cc3_ctx_counters(self.ctx)

    def set_tracing(self, on=True):
        cc3_ctx_set_tracing(self.ctx, on)

    def trace(self):
        return cc3_ctx_trace(self.ctx)

    def _new(self, shape):
        if self.device:
            import torch
            return torch.empty(shape, dtype=torch.float64, device="cuda")
        return np.empty(shape, dtype=np.float64)

    def omega(self, prec=CC3_FP64, out=None):
        """Returns (Omega1, Omega2, E_T) as numpy (host mode) or torch (device)."""
        no, nv = self.no, self.nv
        if out is None:
            out = (self._new((no, nv)), self._new((no, no, nv, nv)), self._new((1,)))
        o1, o2, e = out
        cc3_omega_triples(self.ctx, prec, o1, o2, e, self.stream)
        return o1, o2, e

    def left_jacobian(self, L1, L2, omega, prec=CC3_FP64):
        """Left (transpose) transformation; returns (sigma1, sigma2)."""
        no, nv = self.no, self.nv
        nvec = int(L1.shape[0])
        s1 = self._new((nvec, no, nv))
        s2 = self._new((nvec, no, no, nv, nv))
        cc3_left_jacobian_triples(self.ctx, prec, nvec, omega, L1, L2, s1, s2, self.stream)
        return s1, s2

    def density(self, L1, L2, omega, prec=CC3_FP64):
        """Triples contributions of Algorithm 3 to the one-electron density of
        the left state (L1, L2) at frequency omega; returns (D_oo, D_ov, D_vv)."""
        no, nv = self.no, self.nv
        doo, dov, dvv = self._new((no, no)), self._new((no, nv)), self._new((nv, nv))
        cc3_density_triples(self.ctx, prec, omega, L1, L2, doo, dov, dvv, self.stream)
        return doo, dov, dvv

    def jacobian(self, R1, R2, omega, prec=CC3_FP64):
        no, nv = self.no, self.nv
        nvec = int(R1.shape[0])
        r1 = self._new((nvec, no, nv))
        r2 = self._new((nvec, no, no, nv, nv))
        cc3_jacobian_triples(self.ctx, prec, nvec, omega, R1, R2, r1, r2, self.stream)
        return r1, r2


# ---- serving ----------------------------------------------------------------
def cc3_serve_start(hbm_budget_bytes=0, max_slots=4):
    srv = ctypes.c_void_p()
    _check(lib.cc3_serve_start(ctypes.byref(srv), int(hbm_budget_bytes), int(max_slots)),
           "cc3_serve_start")
    return srv


def cc3_serve_footprint(req):
    b = ctypes.c_size_t(0)
    _check(lib.cc3_serve_footprint(ctypes.byref(req), ctypes.byref(b)), "cc3_serve_footprint")
    return int(b.value)


def cc3_serve_submit(srv, req):
    t = ctypes.c_uint64(0)
    _check(lib.cc3_serve_submit(srv, ctypes.byref(req), ctypes.byref(t)), "cc3_serve_submit")
    return int(t.value)


def cc3_serve_poll(srv, ticket):
    d = ctypes.c_int(0)
    _check(lib.cc3_serve_poll(srv, ctypes.c_uint64(ticket), ctypes.byref(d)), "cc3_serve_poll")
    return bool(d.value)


def cc3_serve_wait(srv, ticket, timeout_s=-1.0):
    """Returns the request's status (raises only for an unknown ticket)."""
    st = lib.cc3_serve_wait(srv, ctypes.c_uint64(ticket), float(timeout_s))
    if st == CC3_ERR_NOT_FOUND:
        _check(st, "cc3_serve_wait")
    return st


def cc3_serve_cancel(srv, ticket):
    _check(lib.cc3_serve_cancel(srv, ctypes.c_uint64(ticket)), "cc3_serve_cancel")


def cc3_serve_stats(srv):
    st = Stats()
    _check(lib.cc3_serve_stats(srv, ctypes.byref(st)), "cc3_serve_stats")
    return {n: getattr(st, n) for n, _ in Stats._fields_}


def cc3_serve_stop(srv):
    _check(lib.cc3_serve_stop(srv), "cc3_serve_stop")


def _f64(x):
    return None if x is None else np.ascontiguousarray(x, dtype=np.float64)


class Server:
    """Owns one cc3_server.  ``submit_omega`` / ``submit_jacobian`` take host
    inputs with the fields of cc3_inputs.CC3Inputs (copied at submit) and
    return a ticket; ``wait`` returns (status, outputs)."""

    def __init__(self, hbm_budget_bytes=0, max_slots=4):
        self.srv = cc3_serve_start(hbm_budget_bytes, max_slots)
        self._out = {}

    def _request(self, kind, prec, inp, nvec=0, omega=None, R1=None, R2=None, flags=0):
        keep = {n: _f64(getattr(inp, n)) for n in ("eps_o", "eps_v", "t2", "g_vvvo", "g_ooov",
                                                   "g_ovov", "F_ov")}
        L = getattr(inp, "chol_L", None)
        keep["chol_L"] = _f64(L)
        keep["omega"], keep["R1"], keep["R2"] = _f64(omega), _f64(R1), _f64(R2)
        r = Request()
        r.kind, r.prec, r.no, r.nv = int(kind), int(prec), int(inp.no), int(inp.nv)
        r.naux = 0 if L is None else int(L.shape[0])
        r.nvec = int(nvec)
        r.flags = int(flags)
        for n, a in keep.items():
            setattr(r, n, None if a is None else a.ctypes.data)
        no, nv = int(inp.no), int(inp.nv)
        if kind == 0:
            out = (np.empty((no, nv)), np.empty((no, no, nv, nv)), np.empty(1))
            r.Omega1, r.Omega2, r.E_T = (o.ctypes.data for o in out)
        else:
            out = (np.empty((nvec, no, nv)), np.empty((nvec, no, no, nv, nv)))
            r.rho1, r.rho2 = (o.ctypes.data for o in out)
        return r, keep, out

    def footprint(self, kind, prec, inp, nvec=0, omega=None, R1=None, R2=None):
        r, _keep, _out = self._request(kind, prec, inp, nvec, omega, R1, R2)
        return cc3_serve_footprint(r)

    def submit_omega(self, inp, prec=CC3_FP64, flags=0):
        r, keep, out = self._request(0, prec, inp, flags=flags)
        t = cc3_serve_submit(self.srv, r)
        self._out[t] = out
        return t

    def submit_jacobian(self, inp, R1, R2, omega, prec=CC3_FP64):
        R1 = _f64(R1)
        nvec = int(R1.shape[0])
        w = np.broadcast_to(np.asarray(omega, dtype=np.float64), (nvec,))
        r, keep, out = self._request(1, prec, inp, nvec, w, R1, R2)
        t = cc3_serve_submit(self.srv, r)
        self._out[t] = out
        return t

    def poll(self, ticket):
        return cc3_serve_poll(self.srv, ticket)

    def wait(self, ticket, timeout_s=-1.0):
        st = cc3_serve_wait(self.srv, ticket, timeout_s)
        if st == CC3_ERR_TIMEOUT:
            return st, None
        return st, self._out.pop(ticket, None)

    def cancel(self, ticket):
        cc3_serve_cancel(self.srv, ticket)

    def stats(self):
        return cc3_serve_stats(self.srv)

    def stop(self):
        if getattr(self, "srv", None):
            cc3_serve_stop(self.srv)
            self.srv = None
            self._out.clear()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
