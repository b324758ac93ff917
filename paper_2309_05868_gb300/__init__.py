"""rand_cholQR on GB300: Python binding of librandqr.so (C ABI in include/randqr.h).

Argument marshalling only: every step of the factorization runs in the library's CUDA
kernels.  Tensors are torch CUDA tensors (float64, row-major, contiguous rows); torch is
used for device memory and streams.  If the library is missing this module raises on
first use -- there is no CPU fallback.

Method: Higgins, Szyld, Boman & Yamazaki, arXiv 2309.05868 (Algorithms 1-4).  Letters: V
is m x n (m rows), sketch sizes s1 (CountSketch) and s2 (Gaussian).
"""
import ctypes as _ct
import os as _os

__all__ = ["RandQRError", "Context", "randqr_cs_hash", "randqr_gauss_sketch", "randqr_rademacher_sketch",
           "randqr_sketch", "SKETCH_GAUSSIAN", "SKETCH_RADEMACHER", "SKETCH_COUNT_ONLY",
           "SKETCH_GAUSSIAN_ONLY",
           "randqr_factor", "randqr_factor_host", "randqr_randqr", "randqr_cholqr2", "randqr_shifted_cholqr3",
           "randqr_shard_sketch", "randqr_sketch_r", "randqr_shard_gram", "randqr_shard_finish",
           "randqr_sketch_static", "randqr_sketch_static_status",
           "default_sketch_sizes", "library_path", "FP64", "F32X2"]

FP64, F32X2 = 0, 1
SKETCH_GAUSSIAN, SKETCH_RADEMACHER, SKETCH_COUNT_ONLY, SKETCH_GAUSSIAN_ONLY = 0, 1, 2, 3
_HERE = _os.path.dirname(_os.path.abspath(__file__))
_LIB_PATH = _os.path.join(_HERE, "_build", "librandqr.so")
_lib = None

_STATUS = {0: "OK", 1: "PENDING", -1: "ERR_ARG", -2: "ERR_NOT_SPD", -3: "ERR_RANK",
           -4: "ERR_NONFINITE", -5: "ERR_NOMEM", -6: "ERR_ADMISSION", -7: "ERR_TIMEOUT",
           -8: "ERR_CUDA", -9: "ERR_TICKET"}


class RandQRError(RuntimeError):
    def __init__(self, status, info=None, detail=""):
        self.status = status
        self.name = _STATUS.get(status, str(status))
        self.info = info
        msg = f"randqr: {self.name}"
        if info is not None and info.info:
            msg += f" (pivot {info.info}, stage {info.stage})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class Info(_ct.Structure):
    _fields_ = [("info", _ct.c_int32), ("stage", _ct.c_int32),
                ("rs_min_diag", _ct.c_double), ("rs_max_diag", _ct.c_double),
                ("want_accuracy", _ct.c_int32), ("reserved", _ct.c_int32),
                ("orth_err2", _ct.c_double), ("resid_relF", _ct.c_double)]


def _info(accuracy=False):
    i = Info()
    i.want_accuracy = 1 if accuracy else 0
    i.orth_err2 = i.resid_relF = -1.0
    return i


def library_path():
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not _os.path.exists(_LIB_PATH):
        raise RuntimeError(f"librandqr.so not built ({_LIB_PATH}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = _ct.CDLL(_LIB_PATH)
    vp, i64, u64, i32 = _ct.c_void_p, _ct.c_int64, _ct.c_uint64, _ct.c_int32
    sig = {
        "randqr_create": [_ct.POINTER(vp), _ct.c_int, _ct.c_size_t],
        "randqr_destroy": [vp],
        "randqr_get_status": [vp, vp, _ct.POINTER(Info)],
        "randqr_cs_hash": [vp, u64, i64, i64, vp, vp, vp],
        "randqr_gauss_sketch": [vp, u64, i64, i64, vp, vp],
        "randqr_rademacher_sketch": [vp, u64, i64, i64, vp, vp],
        "randqr_set_sketch_kind": [vp, i32],
        "randqr_sketch": [vp, vp, i64, i64, i64, i64, i64, u64, vp, vp, vp],
        "randqr_sketch_static": [vp, i64, i64, i64, i64, i64, u64, vp, vp, vp],
        "randqr_sketch_static_status": [vp, _ct.POINTER(Info)],
        "randqr_set_wait_limit": [vp, i32],
        "randqr_factor": [vp, vp, i64, i64, i64, i64, i64, u64, vp, _ct.c_int, vp, i64, vp, i64,
                          _ct.POINTER(Info), vp],
        "randqr_factor_host": [vp, vp, i64, i64, i64, i64, i64, u64, vp, _ct.c_int, vp, i64, vp, i64,
                               _ct.POINTER(Info), vp],
        "randqr_randqr": [vp, vp, i64, i64, i64, i64, i64, u64, vp, vp, i64, vp, i64,
                          _ct.POINTER(Info), vp],
        "randqr_cholqr2": [vp, vp, i64, i64, i64, vp, i64, vp, i64, _ct.POINTER(Info), vp],
        "randqr_shifted_cholqr3": [vp, vp, i64, i64, i64, vp, i64, vp, i64, _ct.POINTER(Info), vp],
        "randqr_shard_sketch": [vp, vp, i64, i64, i64, i64, i64, i64, u64, vp, vp, vp],
        "randqr_sketch_r": [vp, vp, i64, i64, vp, i64, _ct.POINTER(Info), vp],
        "randqr_shard_gram": [vp, vp, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp],
        "randqr_shard_finish": [vp, vp, i64, i64, i64, vp, i64, vp, i64, vp, i64,
                                _ct.POINTER(Info), vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = i32
    L.randqr_status_string.restype = _ct.c_char_p
    L.randqr_status_string.argtypes = [i32]
    L.randqr_last_cuda_error.restype = _ct.c_char_p
    L.randqr_last_cuda_error.argtypes = [vp]
    L.randqr_workspace_bytes.restype = _ct.c_size_t
    L.randqr_workspace_bytes.argtypes = [vp]
    L.randqr_set_profiling.restype = i32
    L.randqr_set_profiling.argtypes = [vp, _ct.c_int]
    L.randqr_get_kernel_times.restype = i32
    L.randqr_get_kernel_times.argtypes = [vp, i32, _ct.POINTER(_ct.c_double),
                                          _ct.POINTER(_ct.c_int64), _ct.POINTER(i32)]
    L.randqr_kernel_name.restype = _ct.c_char_p
    L.randqr_kernel_name.argtypes = [i32]
    _lib = L
    return L


def default_sketch_sizes(n):
    """(s1, s2) = (2 (n^2 + n), 4 n)."""
    return 2 * (n * n + n), 4 * n


class Context:
    """Owns a randqr_ctx (workspace, cached Gaussian sketch, device status word)."""

    def __init__(self, device=0, hbm_budget_bytes=0):
        L = _load()
        self._h = _ct.c_void_p()
        st = L.randqr_create(_ct.byref(self._h), int(device), int(hbm_budget_bytes))
        if st != 0:
            raise RandQRError(st)
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _load().randqr_destroy(self._h)
            self._h = _ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self):
        return int(_load().randqr_workspace_bytes(self._h))

    def set_profiling(self, enable=True):
        self._check(_load().randqr_set_profiling(self._h, int(bool(enable))))

    def set_tensor_cores(self, enable=True):
        """Sketch GEMM, solves and Gram as exact split products on the tensor cores (default), or
        on CUDA cores (FP64 or FP32-pair substitution and Gram)."""
        L = _load()
        L.randqr_set_tensor_cores.argtypes = [_ct.c_void_p, _ct.c_int]
        L.randqr_set_tensor_cores.restype = _ct.c_int32
        self._check(L.randqr_set_tensor_cores(self._h, int(bool(enable))))

    def set_fused_first_pass(self, enable=True):
        """rand_cholQR at n = 64: the first solve and the Gram of W in one launch on paired CTAs,
        or as two passes (the default); see randqr.h."""
        L = _load()
        L.randqr_set_fused_first_pass.argtypes = [_ct.c_void_p, _ct.c_int]
        L.randqr_set_fused_first_pass.restype = _ct.c_int32
        self._check(L.randqr_set_fused_first_pass(self._h, int(bool(enable))))

    def set_wait_limit(self, polls):
        """Poll bound of the kernels' bounded waits (< 0: the defaults); see randqr.h."""
        self._check(_load().randqr_set_wait_limit(self._h, int(polls)))

    def set_sketch_kind(self, kind):
        """The sketch of Algorithm 1 step 1: SKETCH_GAUSSIAN or SKETCH_RADEMACHER multisketch
        (S2 generated when a call passes none), SKETCH_COUNT_ONLY (S2 = I, s2 == s1) or
        SKETCH_GAUSSIAN_ONLY (S1 = I, s1 == m)."""
        self._check(_load().randqr_set_sketch_kind(self._h, int(kind)))

    def kernel_times(self):
        """{kernel name: (total device ms, launches)} recorded since the last read."""
        L = _load()
        tot = (_ct.c_double * 32)()
        cnt = (_ct.c_int64 * 32)()
        nk = _ct.c_int32(0)
        self._check(L.randqr_get_kernel_times(self._h, 32, tot, cnt, _ct.byref(nk)))
        return {L.randqr_kernel_name(k).decode(): (tot[k], int(cnt[k]))
                for k in range(nk.value) if cnt[k]}

    def _check(self, st, info=None):
        if st != 0:
            detail = _load().randqr_last_cuda_error(self._h).decode() if st == -8 else ""
            raise RandQRError(st, info, detail)


_default_ctx = {}


def _ctx(ctx, t):
    if ctx is not None:
        return ctx
    dev = t.device.index if t.device.index is not None else 0
    if dev not in _default_ctx:
        _default_ctx[dev] = Context(dev)
    return _default_ctx[dev]


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return _ct.c_void_p(s.cuda_stream)


def _ptr(t):
    return _ct.c_void_p(t.data_ptr()) if t is not None else None


def _check_mat(t, name):
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.dim() == 2 and t.stride(1) == 1):
        raise ValueError(f"{name}: need a CUDA float64 matrix with unit column stride")
    return t.stride(0)


# ---------------------------------------------------------------------------------------
# Entry points, same names as the C ABI.
# ---------------------------------------------------------------------------------------
def randqr_cs_hash(seed, m, s1, device=0, ctx=None, stream=None):
    """CountSketch buckets (int32) and signs (int8) of rows 0..m-1, on the device."""
    import torch
    bucket = torch.empty(m, dtype=torch.int32, device=f"cuda:{device}")
    sign = torch.empty(m, dtype=torch.int8, device=f"cuda:{device}")
    c = _ctx(ctx, bucket)
    c._check(_load().randqr_cs_hash(c.handle, seed, m, s1, _ptr(bucket), _ptr(sign), _stream(stream)))
    return bucket, sign


def randqr_gauss_sketch(seed, s2, s1, device=0, ctx=None, stream=None):
    """Gaussian sketch S2 (s2 x s1, N(0, 1/s2)) on the device."""
    import torch
    S2 = torch.empty((s2, s1), dtype=torch.float64, device=f"cuda:{device}")
    c = _ctx(ctx, S2)
    c._check(_load().randqr_gauss_sketch(c.handle, seed, s2, s1, _ptr(S2), _stream(stream)))
    return S2


def randqr_rademacher_sketch(seed, s2, s1, device=0, ctx=None, stream=None):
    """Rademacher sketch S2 (s2 x s1, entries +-1/sqrt(s2)) on the device."""
    import torch
    S2 = torch.empty((s2, s1), dtype=torch.float64, device=f"cuda:{device}")
    c = _ctx(ctx, S2)
    c._check(_load().randqr_rademacher_sketch(c.handle, seed, s2, s1, _ptr(S2), _stream(stream)))
    return S2


def randqr_sketch(V, s1, s2, seed=0, S2=None, ctx=None, stream=None):
    """Ws = S2 S1 V (s2 x n)."""
    import torch
    ldv = _check_mat(V, "V")
    m, n = V.shape
    Ws = torch.empty((s2, n), dtype=torch.float64, device=V.device)
    if S2 is not None:
        _check_mat(S2, "S2")
    c = _ctx(ctx, V)
    c._check(_load().randqr_sketch(c.handle, _ptr(V), m, n, ldv, s1, s2, seed, _ptr(S2), _ptr(Ws),
                                   _stream(stream)))
    return Ws


def randqr_sketch_static(V, s1, s2, S2, Ws, seed=0, stream=None):
    """Ws = S2 S1 V through the allocation-free entry point: no context, no device
    allocation (its scratch is a fixed device array, s1 * n <= 2^20).  For callers that
    cannot allocate device memory where they sketch; Ws (s2 x n) and S2 are caller-owned.
    Calls that overlap on the GPU share the scratch and race."""
    ldv = _check_mat(V, "V")
    _check_mat(S2, "S2")
    _check_mat(Ws, "Ws")
    m, n = V.shape
    st = _load().randqr_sketch_static(_ptr(V), m, n, ldv, s1, s2, seed, _ptr(S2), _ptr(Ws),
                                      _stream(stream))
    if st != 0:
        raise RandQRError(st)
    return Ws


def randqr_set_wait_limit(ctx, polls):
    """Poll bound of the kernels' bounded waits on this context (< 0: the defaults); with
    ctx None, the bound of randqr_sketch_static."""
    if ctx is None:
        st = _load().randqr_set_wait_limit(None, int(polls))
        if st != 0:
            raise RandQRError(st)
    else:
        ctx.set_wait_limit(polls)


def randqr_sketch_static_status(stream=None):
    """(status, Info) of the last randqr_sketch_static call on the current device: waits for
    `stream` and reads the fixed status word (no allocation)."""
    info = _info()
    st = _load().randqr_sketch_static_status(_stream(stream), _ct.byref(info))
    return st, info


def _alloc_qr(V, Q, R):
    import torch
    m, n = V.shape
    if Q is None:
        Q = torch.empty((m, n), dtype=torch.float64, device=V.device)
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, device=V.device)
    return Q, R, _check_mat(Q, "Q"), _check_mat(R, "R")


def randqr_factor(V, s1=None, s2=None, seed=0, S2=None, prec=FP64, Q=None, R=None, ctx=None,
                  stream=None, sync=True, accuracy=False):
    """rand_cholQR (Algorithm 3): returns (Q, R, info).  With sync=False the call only
    enqueues work and info is None (read it later with Context.status).  accuracy=True
    (with sync) also measures info.orth_err2 and info.resid_relF on the device."""
    ldv = _check_mat(V, "V")
    m, n = V.shape
    d1, d2 = default_sketch_sizes(n)
    s1 = d1 if s1 is None else s1
    s2 = d2 if s2 is None else s2
    if S2 is not None:
        _check_mat(S2, "S2")
    Q, R, ldq, ldr = _alloc_qr(V, Q, R)
    c = _ctx(ctx, V)
    info = _info(accuracy) if sync else None
    st = _load().randqr_factor(c.handle, _ptr(V), m, n, ldv, s1, s2, seed, _ptr(S2), int(prec),
                               _ptr(Q), ldq, _ptr(R), ldr,
                               _ct.byref(info) if sync else None, _stream(stream))
    c._check(st, info)
    return Q, R, info


def _check_host_mat(t, name):
    import torch
    if not (t.device.type == "cpu" and t.dtype == torch.float64 and t.dim() == 2 and t.stride(1) == 1):
        raise ValueError(f"{name}: need a host float64 matrix with unit column stride")
    return t.stride(0)


def randqr_factor_host(V, s1=None, s2=None, seed=0, S2=None, prec=FP64, Q=None, R=None, ctx=None,
                       device=0, stream=None, sync=True, accuracy=False):
    """rand_cholQR of a host matrix (pinned for asynchronous copies): V is uploaded into the
    context's staging area, factored there in place, and Q and R come back into host
    tensors (allocated pinned when not given).  Returns (Q, R, info); with sync=False only
    enqueued on `stream` (info None): V, Q and R must then stay alive until it completes."""
    import torch
    ldv = _check_host_mat(V, "V")
    m, n = V.shape
    d1, d2 = default_sketch_sizes(n)
    s1 = d1 if s1 is None else s1
    s2 = d2 if s2 is None else s2
    if S2 is not None:
        _check_mat(S2, "S2")
    if Q is None:
        Q = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    ldq, ldr = _check_host_mat(Q, "Q"), _check_host_mat(R, "R")
    c = ctx if ctx is not None else _ctx(None, torch.empty(0, device=f"cuda:{device}"))
    info = _info(accuracy) if sync else None
    st = _load().randqr_factor_host(c.handle, _ptr(V), m, n, ldv, s1, s2, seed, _ptr(S2), int(prec),
                                    _ptr(Q), ldq, _ptr(R), ldr,
                                    _ct.byref(info) if sync else None, _stream(stream))
    c._check(st, info)
    return Q, R, info


def randqr_randqr(V, s1=None, s2=None, seed=0, S2=None, Q=None, R=None, ctx=None, stream=None):
    """randQR (Algorithm 1): returns (Q0, R0, info)."""
    ldv = _check_mat(V, "V")
    m, n = V.shape
    d1, d2 = default_sketch_sizes(n)
    s1 = d1 if s1 is None else s1
    s2 = d2 if s2 is None else s2
    Q, R, ldq, ldr = _alloc_qr(V, Q, R)
    c = _ctx(ctx, V)
    info = Info()
    st = _load().randqr_randqr(c.handle, _ptr(V), m, n, ldv, s1, s2, seed, _ptr(S2), _ptr(Q), ldq,
                               _ptr(R), ldr, _ct.byref(info), _stream(stream))
    c._check(st, info)
    return Q, R, info


def _baseline(fn, V, Q, R, ctx, stream, sync, accuracy=False):
    ldv = _check_mat(V, "V")
    m, n = V.shape
    Q, R, ldq, ldr = _alloc_qr(V, Q, R)
    c = _ctx(ctx, V)
    info = _info(accuracy) if sync else None
    st = fn(c.handle, _ptr(V), m, n, ldv, _ptr(Q), ldq, _ptr(R), ldr,
            _ct.byref(info) if sync else None, _stream(stream))
    c._check(st, info)
    return Q, R, info


def randqr_cholqr2(V, Q=None, R=None, ctx=None, stream=None, sync=True, accuracy=False):
    """CholeskyQR2 (Algorithm 4): returns (Q, R, info)."""
    return _baseline(_load().randqr_cholqr2, V, Q, R, ctx, stream, sync, accuracy)


def randqr_shifted_cholqr3(V, Q=None, R=None, ctx=None, stream=None, sync=True, accuracy=False):
    """Shifted CholeskyQR3: returns (Q, R, info)."""
    return _baseline(_load().randqr_shifted_cholqr3, V, Q, R, ctx, stream, sync, accuracy)


# ---------------------------------------------------------------------------------------
# Row-sharded rand_cholQR (Sec. 4.1): the stages between the two cross-shard sums.
# ---------------------------------------------------------------------------------------
def randqr_shard_sketch(V, row0, s1, s2, seed=0, S2=None, ctx=None, stream=None):
    """Ws_k = S2 S1_k V_k (s2 x n) of a row block whose first row is global row ``row0``."""
    import torch
    ldv = _check_mat(V, "V")
    m, n = V.shape
    Ws = torch.empty((s2, n), dtype=torch.float64, device=V.device)
    if S2 is not None:
        _check_mat(S2, "S2")
    c = _ctx(ctx, V)
    c._check(_load().randqr_shard_sketch(c.handle, _ptr(V), m, n, ldv, int(row0), s1, s2, seed,
                                         _ptr(S2), _ptr(Ws), _stream(stream)))
    return Ws


def randqr_sketch_r(Ws, Rs=None, ctx=None, stream=None, sync=True):
    """R_s (n x n, dense upper) from the summed sketch Ws: returns (Rs, info)."""
    import torch
    _check_mat(Ws, "Ws")
    s2, n = Ws.shape
    if Rs is None:
        Rs = torch.empty((n, n), dtype=torch.float64, device=Ws.device)
    ldr = _check_mat(Rs, "Rs")
    c = _ctx(ctx, Ws)
    info = Info() if sync else None
    st = _load().randqr_sketch_r(c.handle, _ptr(Ws), s2, n, _ptr(Rs), ldr,
                                 _ct.byref(info) if sync else None, _stream(stream))
    c._check(st, info)
    return Rs, info


def randqr_shard_gram(V, Rs, Q=None, G=None, ctx=None, stream=None):
    """W_k = V_k R_s^{-1} (into Q; Q may be V) and G_k = W_k^T W_k: returns (Q, G)."""
    import torch
    ldv = _check_mat(V, "V")
    ldrs = _check_mat(Rs, "Rs")
    m, n = V.shape
    if Q is None:
        Q = torch.empty((m, n), dtype=torch.float64, device=V.device)
    if G is None:
        G = torch.empty((n, n), dtype=torch.float64, device=V.device)
    ldq, ldg = _check_mat(Q, "Q"), _check_mat(G, "G")
    c = _ctx(ctx, V)
    c._check(_load().randqr_shard_gram(c.handle, _ptr(V), m, n, ldv, _ptr(Rs), ldrs, _ptr(Q), ldq,
                                       _ptr(G), ldg, _stream(stream)))
    return Q, G


def randqr_shard_finish(Q, G, Rs, R=None, ctx=None, stream=None, sync=True):
    """R_c = chol(G), Q_k = W_k R_c^{-1} in place, R = R_c R_s: returns (Q, R, info)."""
    import torch
    ldq = _check_mat(Q, "Q")
    ldg, ldrs = _check_mat(G, "G"), _check_mat(Rs, "Rs")
    m, n = Q.shape
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, device=Q.device)
    ldr = _check_mat(R, "R")
    c = _ctx(ctx, Q)
    info = Info() if sync else None
    st = _load().randqr_shard_finish(c.handle, _ptr(Q), m, n, ldq, _ptr(G), ldg, _ptr(Rs), ldrs,
                                     _ptr(R), ldr, _ct.byref(info) if sync else None,
                                     _stream(stream))
    c._check(st, info)
    return Q, R, info


def get_status(ctx, stream=None):
    """Wait for `stream` and return (status, Info) of the context's last call."""
    info = Info()
    st = _load().randqr_get_status(ctx.handle, _stream(stream), _ct.byref(info))
    return st, info


# ---------------------------------------------------------------------------------------
# Serving: randqr_submit / randqr_poll (continuous batching over the context's slots).
# ---------------------------------------------------------------------------------------
ALGO_RAND_CHOLQR, ALGO_CHOLQR2, ALGO_SHIFTED_CHOLQR3 = 0, 1, 2
PENDING = 1


class Request(_ct.Structure):
    _fields_ = [("algo", _ct.c_int32), ("prec", _ct.c_int32), ("V", _ct.c_void_p),
                ("m", _ct.c_int64), ("n", _ct.c_int64), ("ldv", _ct.c_int64),
                ("s1", _ct.c_int64), ("s2", _ct.c_int64), ("seed", _ct.c_uint64),
                ("Q", _ct.c_void_p), ("ldq", _ct.c_int64), ("R", _ct.c_void_p),
                ("ldr", _ct.c_int64), ("max_orth_err", _ct.c_double),
                ("want_accuracy", _ct.c_int32), ("reserved", _ct.c_int32)]


class ServeStats(_ct.Structure):
    _fields_ = [("submitted", _ct.c_uint64), ("completed", _ct.c_uint64),
                ("queued", _ct.c_uint64), ("running", _ct.c_uint64),
                ("bytes_in_flight", _ct.c_size_t), ("slots", _ct.c_int32),
                ("budget", _ct.c_size_t)]


def _serve_sigs(L):
    if getattr(L, "_serve_ready", False):
        return L
    vp, i32 = _ct.c_void_p, _ct.c_int32
    for name, args in {
        "randqr_serve_config": [vp, i32, _ct.c_size_t],
        "randqr_submit": [vp, _ct.POINTER(Request), _ct.POINTER(_ct.c_uint64)],
        "randqr_submit_batch": [vp, _ct.POINTER(Request), i32, _ct.POINTER(_ct.c_uint64)],
        "randqr_poll": [vp, _ct.c_uint64, _ct.POINTER(Info)],
        "randqr_wait": [vp, _ct.c_uint64, _ct.POINTER(Info)],
        "randqr_serve_stats_get": [vp, _ct.POINTER(ServeStats)],
    }.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = i32
    L._serve_ready = True
    return L


_inflight = {}  # (context handle, ticket) -> tensors kept alive until the ticket retires


def make_request(V, Q=None, R=None, algo=ALGO_RAND_CHOLQR, prec=FP64, s1=0, s2=0, seed=0,
                 max_orth_err=0.0, accuracy=False):
    """A randqr_request over torch tensors (Q, R allocated if not given)."""
    ldv = _check_mat(V, "V")
    Q, R, ldq, ldr = _alloc_qr(V, Q, R)
    m, n = V.shape
    r = Request(algo, prec, V.data_ptr(), m, n, ldv, s1, s2, seed, Q.data_ptr(), ldq,
                R.data_ptr(), ldr, max_orth_err, 1 if accuracy else 0, 0)
    return r, (V, Q, R)


def randqr_serve_config(ctx, slots=8, hbm_budget_bytes=0):
    ctx._check(_serve_sigs(_load()).randqr_serve_config(ctx.handle, slots, hbm_budget_bytes))


def randqr_submit(ctx, V, Q=None, R=None, **kw):
    """Submit one request; returns (ticket, (V, Q, R))."""
    L = _serve_sigs(_load())
    req, keep = make_request(V, Q, R, **kw)
    t = _ct.c_uint64(0)
    st = L.randqr_submit(ctx.handle, _ct.byref(req), _ct.byref(t))
    if st != 0:
        raise RandQRError(st)
    _inflight[(ctx.handle.value, t.value)] = keep
    return t.value, keep


def randqr_submit_batch(ctx, requests):
    """requests: list of (Request, keep) from make_request; returns the tickets."""
    L = _serve_sigs(_load())
    arr = (Request * len(requests))(*[r for r, _ in requests])
    tickets = (_ct.c_uint64 * len(requests))()
    st = L.randqr_submit_batch(ctx.handle, arr, len(requests), tickets)
    if st != 0:
        raise RandQRError(st)
    for (r, keep), t in zip(requests, tickets):
        _inflight[(ctx.handle.value, t)] = keep
    return list(tickets)


def _retire(ctx, ticket, st):
    if st != PENDING:
        _inflight.pop((ctx.handle.value, ticket), None)


def randqr_poll(ctx, ticket):
    """(status, Info): status 1 (PENDING) while queued or running."""
    info = Info()
    st = _serve_sigs(_load()).randqr_poll(ctx.handle, ticket, _ct.byref(info))
    _retire(ctx, ticket, st)
    return st, info


def randqr_wait(ctx, ticket):
    info = Info()
    st = _serve_sigs(_load()).randqr_wait(ctx.handle, ticket, _ct.byref(info))
    _retire(ctx, ticket, st)
    return st, info


def randqr_serve_stats_get(ctx):
    s = ServeStats()
    ctx._check(_serve_sigs(_load()).randqr_serve_stats_get(ctx.handle, _ct.byref(s)))
    return {f: getattr(s, f) for f, _ in ServeStats._fields_}


# ---------------------------------------------------------------------------------------
# Batched: randqr_factor_batched (one CUDA graph per batch, autotuned lane count).
# ---------------------------------------------------------------------------------------
class BatchItem(_ct.Structure):
    _fields_ = [("V", _ct.c_void_p), ("m", _ct.c_int64), ("n", _ct.c_int64), ("ldv", _ct.c_int64),
                ("Q", _ct.c_void_p), ("ldq", _ct.c_int64), ("R", _ct.c_void_p), ("ldr", _ct.c_int64),
                ("s1", _ct.c_int64), ("s2", _ct.c_int64), ("seed", _ct.c_uint64)]


def _batch_sigs(L):
    if getattr(L, "_batch_ready", False):
        return L
    L.randqr_factor_batched.argtypes = [_ct.c_void_p, _ct.POINTER(BatchItem), _ct.c_int32, _ct.c_int,
                                        _ct.POINTER(_ct.c_int32), _ct.c_void_p]
    L.randqr_factor_batched.restype = _ct.c_int32
    L.randqr_batch_plan_info.argtypes = [_ct.c_void_p, _ct.POINTER(BatchItem), _ct.c_int32, _ct.c_int,
                                         _ct.POINTER(_ct.c_int32), _ct.POINTER(_ct.c_float)]
    L.randqr_batch_plan_info.restype = _ct.c_int32
    L._batch_ready = True
    return L


def batch_items(Vs, Qs, Rs, seeds=None):
    """The descriptor array for lists of V, Q, R tensors (same order)."""
    arr = (BatchItem * len(Vs))()
    for i, (V, Q, R) in enumerate(zip(Vs, Qs, Rs)):
        ldv, ldq, ldr = _check_mat(V, "V"), _check_mat(Q, "Q"), _check_mat(R, "R")
        m, n = V.shape
        arr[i] = BatchItem(V.data_ptr(), m, n, ldv, Q.data_ptr(), ldq, R.data_ptr(), ldr, 0, 0,
                           0 if seeds is None else int(seeds[i]))
    return arr


def randqr_factor_batched(ctx, items, prec=FP64, stream=None, sync=True):
    """Factor every item of `items` (from batch_items); returns the per-item statuses when
    sync, else None.  The first call with a given array builds and autotunes its graph."""
    L = _batch_sigs(_load())
    n = len(items)
    st_arr = (_ct.c_int32 * n)() if sync else None
    st = L.randqr_factor_batched(ctx.handle, items, n, int(prec), st_arr, _stream(stream))
    if st not in (0, -2, -3) or (st != 0 and not sync):
        raise RandQRError(st)
    return list(st_arr) if sync else None


def randqr_batch_plan_info(ctx, items, prec=FP64):
    L = _batch_sigs(_load())
    lanes, ms = _ct.c_int32(0), _ct.c_float(0)
    st = L.randqr_batch_plan_info(ctx.handle, items, len(items), int(prec), _ct.byref(lanes), _ct.byref(ms))
    if st != 0:
        raise RandQRError(st)
    return lanes.value, ms.value
