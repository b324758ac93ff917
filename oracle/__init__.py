"""CPU oracle for rand_cholQR (arXiv 2309.05868) -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may import this
package.  It is a thin ctypes wrapper over ``oracle.c`` (plain FP64 C, row-major) and
shares no code with the CUDA library.  Letters: V is m x n (m rows), sketch sizes s1, s2.

Functions return numpy arrays; numerical failures raise ``OracleError`` with the status
code (-2 Cholesky breakdown with ``info`` = 1-based pivot, -3 zero diagonal in R).
"""
import ctypes as _ct
import numpy as _np

from . import build as _build

_lib = None

_D = _ct.POINTER(_ct.c_double)
_I64 = _ct.c_int64
_U64 = _ct.c_uint64


class OracleError(RuntimeError):
    def __init__(self, status, info=0):
        super().__init__(f"oracle status {status} (info {info})")
        self.status = status
        self.info = info


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = _ct.CDLL(_build.build())
    lib.orc_splitmix64.restype = _U64
    lib.orc_splitmix64.argtypes = [_U64]
    lib.orc_cs_hash.argtypes = [_U64, _I64, _I64, _ct.POINTER(_ct.c_int32), _ct.POINTER(_ct.c_int8)]
    lib.orc_philox4x64_10.argtypes = [_ct.POINTER(_U64), _ct.POINTER(_U64), _ct.POINTER(_U64)]
    lib.orc_gauss_sketch.argtypes = [_U64, _I64, _I64, _D]
    lib.orc_rademacher_sketch.argtypes = [_U64, _I64, _I64, _D]
    lib.orc_countsketch.argtypes = [_D, _I64, _I64, _I64, _I64, _U64, _D]
    lib.orc_countsketch_rows.argtypes = [_D, _I64, _I64, _I64, _I64, _U64, _I64, _D]
    lib.orc_cs_hash_at.argtypes = [_U64, _I64, _I64, _I64, _ct.POINTER(_ct.c_int32),
                                   _ct.POINTER(_ct.c_int8)]
    lib.orc_gemm.argtypes = [_D, _D, _I64, _I64, _I64, _D]
    lib.orc_hhqr_r.argtypes = [_D, _I64, _I64, _D]
    lib.orc_householder_qr.argtypes = [_D, _I64, _I64, _I64, _D, _D]
    lib.orc_trsm.argtypes = [_D, _I64, _I64, _I64, _D, _D, _I64]
    lib.orc_gram.argtypes = [_D, _I64, _I64, _I64, _D]
    lib.orc_chol.argtypes = [_D, _I64, _D, _ct.POINTER(_ct.c_int32)]
    lib.orc_trmm.argtypes = [_D, _D, _I64, _D]
    lib.orc_randqr.argtypes = [_D, _I64, _I64, _I64, _I64, _I64, _U64, _D, _D, _D, _D, _D]
    lib.orc_cholqr.argtypes = [_D, _I64, _I64, _I64, _D, _D, _ct.POINTER(_ct.c_int32)]
    lib.orc_rand_cholqr.argtypes = [_D, _I64, _I64, _I64, _I64, _I64, _U64, _D, _D, _D, _D, _D,
                                    _ct.POINTER(_ct.c_int32)]
    lib.orc_cholqr2.argtypes = [_D, _I64, _I64, _I64, _D, _D, _ct.POINTER(_ct.c_int32)]
    lib.orc_scholqr3.argtypes = [_D, _I64, _I64, _I64, _D, _D, _D, _ct.POINTER(_ct.c_int32)]
    lib.orc_sym_absmax_eig.restype = _ct.c_double
    lib.orc_sym_absmax_eig.argtypes = [_D, _I64]
    lib.orc_orth_err.argtypes = [_D, _I64, _I64, _I64, _D, _D]
    lib.orc_resid.restype = _ct.c_double
    lib.orc_resid.argtypes = [_D, _I64, _I64, _I64, _D, _I64, _D]
    for name in ("orc_countsketch", "orc_countsketch_rows", "orc_hhqr_r", "orc_householder_qr", "orc_chol",
                 "orc_randqr", "orc_cholqr", "orc_rand_cholqr", "orc_cholqr2", "orc_scholqr3"):
        getattr(lib, name).restype = _ct.c_int
    _lib = lib
    return lib


def _p(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a):
    return _np.ascontiguousarray(a, dtype=_np.float64)


def _check(st, info=0):
    if st != 0:
        raise OracleError(st, int(info))


# ---- generators ------------------------------------------------------------------
def splitmix64(x: int) -> int:
    return int(_load().orc_splitmix64(_U64(x & 0xFFFFFFFFFFFFFFFF)))


def cs_hash(seed: int, m: int, s1: int):
    """CountSketch buckets (int32, in [0, s1)) and signs (int8, +-1) for rows 0..m-1."""
    b = _np.empty(m, dtype=_np.int32)
    s = _np.empty(m, dtype=_np.int8)
    _load().orc_cs_hash(_U64(seed), m, s1, b.ctypes.data_as(_ct.POINTER(_ct.c_int32)),
                        s.ctypes.data_as(_ct.POINTER(_ct.c_int8)))
    return b, s


def philox4x64_10(ctr, key):
    c = (_U64 * 4)(*[int(v) & 0xFFFFFFFFFFFFFFFF for v in ctr])
    k = (_U64 * 2)(*[int(v) & 0xFFFFFFFFFFFFFFFF for v in key])
    o = (_U64 * 4)()
    _load().orc_philox4x64_10(c, k, o)
    return [int(v) for v in o]


def gauss_sketch(seed: int, s2: int, s1: int):
    S2 = _np.empty((s2, s1), dtype=_np.float64)
    _load().orc_gauss_sketch(_U64(seed), s2, s1, _p(S2))
    return S2


def rademacher_sketch(seed: int, s2: int, s1: int):
    """Rademacher S2 (s2 x s1) with entries +-1/sqrt(s2) from splitmix64 sign words."""
    S2 = _np.empty((s2, s1), dtype=_np.float64)
    _load().orc_rademacher_sketch(_U64(seed), s2, s1, _p(S2))
    return S2


# ---- steps -----------------------------------------------------------------------
def countsketch(V, s1: int, seed: int):
    V = _f64(V)
    m, n = V.shape
    W1 = _np.empty((s1, n), dtype=_np.float64)
    _check(_load().orc_countsketch(_p(V), m, n, n, s1, _U64(seed), _p(W1)))
    return W1


def countsketch_rows(V, s1: int, seed: int, row0: int):
    """S1_k V_k for a row block whose first row is global row ``row0`` (Sec. 4.1)."""
    V = _f64(V)
    m, n = V.shape
    W1 = _np.empty((s1, n), dtype=_np.float64)
    _check(_load().orc_countsketch_rows(_p(V), m, n, n, s1, _U64(seed), _I64(row0), _p(W1)))
    return W1


def cs_hash_at(seed: int, row0: int, m: int, s1: int):
    """CountSketch buckets and signs of global rows row0 .. row0 + m - 1."""
    b = _np.empty(m, dtype=_np.int32)
    s = _np.empty(m, dtype=_np.int8)
    _load().orc_cs_hash_at(_U64(seed), _I64(row0), m, s1,
                           b.ctypes.data_as(_ct.POINTER(_ct.c_int32)),
                           s.ctypes.data_as(_ct.POINTER(_ct.c_int8)))
    return b, s


def gemm(A, B):
    A, B = _f64(A), _f64(B)
    C = _np.empty((A.shape[0], B.shape[1]), dtype=_np.float64)
    _load().orc_gemm(_p(A), _p(B), A.shape[0], A.shape[1], B.shape[1], _p(C))
    return C


def hhqr_r(A):
    A = _f64(A)
    R = _np.empty((A.shape[1], A.shape[1]), dtype=_np.float64)
    _check(_load().orc_hhqr_r(_p(A), A.shape[0], A.shape[1], _p(R)))
    return R


def householder_qr(V):
    V = _f64(V)
    m, n = V.shape
    Q = _np.empty((m, n), dtype=_np.float64)
    R = _np.empty((n, n), dtype=_np.float64)
    _check(_load().orc_householder_qr(_p(V), m, n, n, _p(Q), _p(R)))
    return Q, R


def trsm(V, R):
    V, R = _f64(V), _f64(R)
    W = _np.empty_like(V)
    _load().orc_trsm(_p(V), V.shape[0], V.shape[1], V.shape[1], _p(R), _p(W), V.shape[1])
    return W


def gram(W):
    W = _f64(W)
    G = _np.empty((W.shape[1], W.shape[1]), dtype=_np.float64)
    _load().orc_gram(_p(W), W.shape[0], W.shape[1], W.shape[1], _p(G))
    return G


def chol(G):
    G = _f64(G)
    n = G.shape[0]
    R = _np.empty((n, n), dtype=_np.float64)
    info = _ct.c_int32(0)
    _check(_load().orc_chol(_p(G), n, _p(R), _ct.byref(info)), info.value)
    return R


def trmm(A, B):
    A, B = _f64(A), _f64(B)
    C = _np.empty_like(A)
    _load().orc_trmm(_p(A), _p(B), A.shape[0], _p(C))
    return C


# ---- algorithms ------------------------------------------------------------------
def randqr(V, s1: int, s2: int, seed: int, S2=None):
    """Algorithm 1.  Returns (Q0, R0, W1, Ws)."""
    V = _f64(V)
    m, n = V.shape
    S2 = None if S2 is None else _f64(S2)
    Q0 = _np.empty((m, n)); R0 = _np.empty((n, n))
    W1 = _np.empty((s1, n)); Ws = _np.empty((s2, n))
    _check(_load().orc_randqr(_p(V), m, n, n, s1, s2, _U64(seed), _p(S2), _p(Q0), _p(R0),
                              _p(W1), _p(Ws)))
    return Q0, R0, W1, Ws


def rand_cholqr(V, s1: int, s2: int, seed: int, S2=None, return_factors=False):
    """Algorithm 3.  Returns (Q, R) or (Q, R, Rs, Rc)."""
    V = _f64(V)
    m, n = V.shape
    S2 = None if S2 is None else _f64(S2)
    Q = _np.empty((m, n)); R = _np.empty((n, n)); Rs = _np.empty((n, n)); Rc = _np.empty((n, n))
    info = _ct.c_int32(0)
    st = _load().orc_rand_cholqr(_p(V), m, n, n, s1, s2, _U64(seed), _p(S2), _p(Q), _p(R),
                                 _p(Rs), _p(Rc), _ct.byref(info))
    _check(st, info.value)
    return (Q, R, Rs, Rc) if return_factors else (Q, R)


def _two_out(fn, V):
    V = _f64(V)
    m, n = V.shape
    Q = _np.empty((m, n)); R = _np.empty((n, n))
    info = _ct.c_int32(0)
    _check(fn(_p(V), m, n, n, _p(Q), _p(R), _ct.byref(info)), info.value)
    return Q, R


def cholqr(V):
    return _two_out(_load().orc_cholqr, V)


def cholqr2(V):
    return _two_out(_load().orc_cholqr2, V)


def scholqr3(V, return_r0=False):
    """Shifted CholeskyQR3.  Returns (Q, R) or (Q, R, R0), R0 the shifted pass's factor."""
    V = _f64(V)
    m, n = V.shape
    Q = _np.empty((m, n)); R = _np.empty((n, n)); R0 = _np.empty((n, n))
    info = _ct.c_int32(0)
    _check(_load().orc_scholqr3(_p(V), m, n, n, _p(Q), _p(R), _p(R0), _ct.byref(info)), info.value)
    return (Q, R, R0) if return_r0 else (Q, R)


# ---- error measures --------------------------------------------------------------
def sym_absmax_eig(A):
    A = _f64(A)
    return float(_load().orc_sym_absmax_eig(_p(A), A.shape[0]))


def orth_err(Q):
    """(||I - Q^T Q||_2, ||I - Q^T Q||_F)."""
    Q = _f64(Q)
    e2 = _ct.c_double(); eF = _ct.c_double()
    _load().orc_orth_err(_p(Q), Q.shape[0], Q.shape[1], Q.shape[1], _ct.byref(e2), _ct.byref(eF))
    return e2.value, eF.value


def resid(V, Q, R):
    """||V - Q R||_F / ||V||_F (R upper triangular)."""
    V, Q, R = _f64(V), _f64(Q), _f64(R)
    return float(_load().orc_resid(_p(V), V.shape[0], V.shape[1], V.shape[1], _p(Q),
                                   Q.shape[1], _p(R)))
