"""Python binding of libpssd: structure-preserving spectral divide-and-conquer
for definite pseudosymmetric matrices on GB300 (arXiv 2203.08900).

Argument marshalling only.  Every step of the computation runs in the CUDA
library behind the C ABI of ``include/pssd.h``; torch supplies device memory
and the current stream.  There is no fallback: if the compiled library is
missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpssd.so")

PSSD_FP64 = 0
PSSD_MIXED = 1
PSSD_FP64_EMULATED = 2
FLAG_RESIDUALS = 1

# kinds reported by profile_read (PSSD_KIND_* of include/pssd.h)
K_DGEMM, K_POTRF, K_HBM, K_GEMV, K_JACOBI, K_SGEMM, K_DFGEMM, K_TCGEMM, K_OZGEMM, K_OZPREP, K_TCPREP = range(11)
KIND_NAMES = ["dgemm", "chol_leaf", "hbm_pass", "gemv", "jacobi_leaf", "sgemm", "dfgemm", "tcgemm", "ozgemm",
              "ozprep", "tcprep"]
FLAG_NO_TENSOR_CORES = 2
FLAG_EMU_SIMT = 4
FLAG_NO_REFINE = 8
FLAG_RECOMPUTE = 16
METHOD_ZOLO, METHOD_DWH, METHOD_NEWTON = 0, 1, 2


class Opts(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("precision", ctypes.c_int), ("max_restarts", ctypes.c_int), ("leaf", ctypes.c_int),
                ("flags", ctypes.c_int), ("method", ctypes.c_int), ("wait_cycles", ctypes.c_longlong)]


class Info(ctypes.Structure):
    _fields_ = [("r_used", ctypes.c_int * 4), ("passes", ctypes.c_int), ("steps", ctypes.c_int),
                ("restarts", ctypes.c_int), ("p", ctypes.c_int), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("ell", ctypes.c_double * 6), ("stop_crit", ctypes.c_double * 4),
                ("s2_resid", ctypes.c_double), ("jsym_resid", ctypes.c_double),
                ("split_backerr", ctypes.c_double), ("fail_index", ctypes.c_int), ("levels", ctypes.c_int),
                ("seconds", ctypes.c_double), ("precision", ctypes.c_int), ("fp32_steps", ctypes.c_int),
                ("ns_steps", ctypes.c_int), ("ns_resid", ctypes.c_double), ("comm_resid", ctypes.c_double),
                ("method", ctypes.c_int), ("iterations", ctypes.c_int)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


class PssdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("pssd status %d: %s" % (status, msg))
        self.status = status


_lib = None

# C-ABI symbols declared in include/pssd.h plus the measurement hooks
EXPORTS = ["pssd_opts_init", "pssd_create", "pssd_destroy", "pssd_set_stream", "pssd_last_cuda_error",
           "pssd_status_string", "pssd_zolo_coeffs", "pssd_choose_r", "pssd_sign", "pssd_split", "pssd_eig",
           "pssd_profile_enable", "pssd_profile_reset", "pssd_profile_read", "pssd_launch_count",
           "pssd_sign_noalloc", "pssd_sign_vjp", "pssd_eig_batched", "pssd_test_gemm_f32",
           "pssd_test_gemm_f64", "pssd_workspace_bytes", "pssd_set_workspace", "pssd_workspace_peak",
           "pssd_device_alloc_count", "pssd_casida_sign", "pssd_casida_split", "pssd_casida_eig",
           "pssd_test_sym_eig", "pssd_sign_vjp_rev", "pssd_zsign", "pssd_zeig", "pssd_launch_count_phases",
           "pssd_test_krylov", "pssd_gsign", "pssd_gsplit"]
NOALLOC_MAX_N = 128
MAX_N = 65535                 # PSSD_MAX_N: largest supported order


def lib():
    """Load libpssd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libpssd.so not built (%s); run paper_2203_08900_gb300.build.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip, cp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_char_p
    L.pssd_opts_init.argtypes = [ctypes.POINTER(Opts)]
    L.pssd_opts_init.restype = None
    L.pssd_create.argtypes = [ctypes.POINTER(vp), vp]
    L.pssd_destroy.argtypes = [vp]
    L.pssd_set_stream.argtypes = [vp, vp]
    L.pssd_last_cuda_error.argtypes = [vp]
    L.pssd_last_cuda_error.restype = cp
    L.pssd_status_string.argtypes = [ctypes.c_int]
    L.pssd_status_string.restype = cp
    L.pssd_zolo_coeffs.argtypes = [ctypes.c_double, ctypes.c_int, dp, dp, dp, dp]
    L.pssd_choose_r.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
    sig = [vp, ctypes.c_int, vp, vp, ctypes.c_int]
    L.pssd_sign.argtypes = sig + [vp, ctypes.c_int, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    L.pssd_split.argtypes = sig + [vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int, ip,
                                   ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    L.pssd_eig.argtypes = sig + [vp, ctypes.c_int, vp, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    L.pssd_sign_noalloc.argtypes = sig + [vp, ctypes.c_int, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    L.pssd_sign_vjp.argtypes = sig + [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.POINTER(Opts),
                                      ctypes.POINTER(Info)]
    L.pssd_sign_vjp_rev.argtypes = sig + [vp, ctypes.c_int, ctypes.c_double, vp, ctypes.c_int, ctypes.POINTER(Opts),
                                          ctypes.POINTER(Info)]
    L.pssd_zsign.argtypes = sig + [vp, ctypes.c_int, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    L.pssd_gsign.argtypes = sig + [vp, ctypes.c_int, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    L.pssd_gsplit.argtypes = sig + [vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int, vp,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    L.pssd_zeig.argtypes = sig + [vp, ctypes.c_int, vp, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    ll = ctypes.c_longlong
    L.pssd_test_gemm_f32.argtypes = [vp] + [ctypes.c_int] * 10 + [ctypes.c_double, ctypes.c_double,
                                     vp, ll, ll, vp, ll, ll, vp, ll, ll, vp, ll, ll, vp]
    L.pssd_test_gemm_f64.argtypes = L.pssd_test_gemm_f32.argtypes
    L.pssd_eig_batched.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(Opts),
                                   ctypes.POINTER(Info)]
    L.pssd_profile_enable.argtypes = [vp, ctypes.c_int]
    L.pssd_profile_reset.argtypes = [vp]
    L.pssd_profile_read.argtypes = [vp, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_longlong), dp, dp]
    L.pssd_launch_count.argtypes = [vp]
    L.pssd_launch_count.restype = ctypes.c_longlong
    cas = [vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int]
    L.pssd_casida_sign.argtypes = cas + [vp, ctypes.c_int, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    L.pssd_casida_split.argtypes = cas + [vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int,
                                          ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    L.pssd_casida_eig.argtypes = cas + [vp, ctypes.c_int, vp, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    L.pssd_test_sym_eig.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.POINTER(Opts),
                                    ctypes.POINTER(Info)]
    L.pssd_device_alloc_count.argtypes = []
    L.pssd_device_alloc_count.restype = ctypes.c_longlong
    L.pssd_launch_count_phases.argtypes = [vp, ctypes.c_int]
    L.pssd_test_krylov.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_ulonglong, ctypes.c_int, vp, vp]
    L.pssd_workspace_bytes.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_size_t)]
    L.pssd_set_workspace.argtypes = [vp, vp, ctypes.c_size_t]
    L.pssd_workspace_peak.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    _lib = L
    return L


def device_alloc_count() -> int:
    """Device allocations (cudaMalloc calls) the library has made in this process."""
    return int(lib().pssd_device_alloc_count())


PHASES = ["other", "front", "bounds", "sign", "split", "shift", "node_sign", "node_split", "assemble", "leaf",
          "refine"]


def launch_count_phases() -> dict:
    """Kernels launched by the library in this process, by phase of the solve (PSSD_PHASE_*)."""
    L = lib()
    n = L.pssd_launch_count_phases(None, 0)
    buf = (ctypes.c_longlong * n)()
    L.pssd_launch_count_phases(buf, n)
    return {PHASES[i] if i < len(PHASES) else str(i): int(buf[i]) for i in range(n)}


def zolo_coeffs(ell: float, r: int):
    """Zolotarev coefficients from the library (host routine)."""
    import numpy as np
    c = (ctypes.c_double * (2 * r))(); a = (ctypes.c_double * r)()
    ch = ctypes.c_double(); l1 = ctypes.c_double()
    st = lib().pssd_zolo_coeffs(float(ell), int(r), c, a, ctypes.byref(ch), ctypes.byref(l1))
    if st:
        raise PssdError(st, "invalid argument")
    return np.array(c[:]), np.array(a[:]), ch.value, l1.value


def choose_r(ell: float, tau: float = 1e-15, r_max: int = 8) -> int:
    st = lib().pssd_choose_r(float(ell), float(tau), int(r_max))
    if st < 0:
        raise PssdError(st, "invalid argument")
    return st


class Handle:
    """Owns a pssd handle bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream: torch.cuda.Stream | None = None):
        L = lib()
        self._h = ctypes.c_void_p()
        s = (stream or torch.cuda.current_stream()).cuda_stream
        st = L.pssd_create(ctypes.byref(self._h), ctypes.c_void_p(s))
        if st:
            raise PssdError(st, "pssd_create failed")

    def close(self):
        if self._h:
            lib().pssd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: torch.cuda.Stream):
        lib().pssd_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream))

    # ---- measurement hooks
    def profile(self, on: bool = True):
        lib().pssd_profile_enable(self._h, 1 if on else 0)

    def profile_reset(self):
        lib().pssd_profile_reset(self._h)

    def profile_read(self, kind: int):
        ms = ctypes.c_double(); cnt = ctypes.c_longlong(); fl = ctypes.c_double(); by = ctypes.c_double()
        lib().pssd_profile_read(self._h, int(kind), ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(fl),
                                ctypes.byref(by))
        return {"ms": ms.value, "launches": cnt.value, "flops": fl.value, "bytes": by.value}

    def launch_count(self) -> int:
        return int(lib().pssd_launch_count(self._h))

    # ---- workspace
    def workspace_bytes(self, n: int, **kw) -> int:
        """pssd_workspace_bytes: upper bound for one sign/split/eig call of order n."""
        b = ctypes.c_size_t(0)
        o = _opts(**kw)
        self._check(lib().pssd_workspace_bytes(self._h, int(n), ctypes.byref(o), ctypes.byref(b)))
        return int(b.value)

    def set_workspace(self, buf: torch.Tensor | None):
        """pssd_set_workspace: use a caller-owned CUDA tensor's memory as the only
        workspace (None: back to library-managed).  The tensor is kept alive here."""
        if buf is None:
            self._check(lib().pssd_set_workspace(self._h, None, 0))
            self._ws = None
            return
        nbytes = buf.numel() * buf.element_size()
        self._check(lib().pssd_set_workspace(self._h, ctypes.c_void_p(buf.data_ptr()), nbytes))
        self._ws = buf

    def workspace_peak(self) -> int:
        b = ctypes.c_size_t(0)
        self._check(lib().pssd_workspace_peak(self._h, ctypes.byref(b)))
        return int(b.value)

    def _check(self, st):
        if st:
            L = lib()
            msg = L.pssd_status_string(st).decode()
            if st in (6, 7):
                msg += " (" + L.pssd_last_cuda_error(self._h).decode() + ")"
            raise PssdError(st, msg)


def _opts(r=0, alpha=0.0, beta=0.0, precision=PSSD_FP64, max_restarts=2, leaf=64, flags=0, method=METHOD_ZOLO,
          wait_cycles=0):
    o = Opts()
    lib().pssd_opts_init(ctypes.byref(o))
    o.r = int(r); o.alpha = float(alpha); o.beta = float(beta); o.precision = int(precision)
    o.max_restarts = int(max_restarts); o.leaf = int(leaf); o.flags = int(flags)
    o.method = int(method); o.wait_cycles = int(wait_cycles)
    return o


def _sigma(n, sigma):
    if sigma is None:
        return None, None
    import numpy as np
    s = np.ascontiguousarray(np.asarray(sigma).astype(np.int8).ravel())
    if s.shape[0] != n:
        raise ValueError("sigma must have n entries")
    return s, s.ctypes.data_as(ctypes.c_void_p)


def _check_H(H):
    if not (isinstance(H, torch.Tensor) and H.is_cuda and H.dtype == torch.float64 and H.dim() == 2
            and H.shape[0] == H.shape[1] and H.stride(1) == 1):
        raise ValueError("H must be a square row-major float64 CUDA tensor")
    return H.shape[0], H.stride(0)


_default = {}


def _handle(handle):
    if handle is not None:
        return handle
    dev = torch.cuda.current_device()
    h = _default.get(dev)
    if h is None:
        h = _default[dev] = Handle()
    h.set_stream(torch.cuda.current_stream())
    return h


def sign(H, sigma=None, handle=None, **kw):
    """S = sign(H).  Returns (S, info dict)."""
    n, ldh = _check_H(H)
    h = _handle(handle)
    S = torch.empty_like(H)
    keep, sp = _sigma(n, sigma)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_sign(h._h, n, sp, ctypes.c_void_p(H.data_ptr()), ldh, ctypes.c_void_p(S.data_ptr()),
                         S.stride(0), ctypes.byref(o), ctypes.byref(info))
    h._check(st)
    return S, info.as_dict()


def gsign(H, sigma=None, handle=None, **kw):
    """S = sign(H) of a general (not necessarily definite) pseudosymmetric H (float64
    CUDA tensor; Sigma H symmetric): scaled Newton on Sigma X.  Returns (S, info dict)."""
    n, ldh = _check_H(H)
    h = _handle(handle)
    S = torch.empty_like(H)
    keep, sp = _sigma(n, sigma)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_gsign(h._h, n, sp, ctypes.c_void_p(H.data_ptr()), ldh, ctypes.c_void_p(S.data_ptr()),
                          S.stride(0), ctypes.byref(o), ctypes.byref(info))
    h._check(st)
    return S, info.as_dict()


def gsplit(H, sigma=None, handle=None, **kw):
    """Spectral division of a general pseudosymmetric H (float64 CUDA tensor).  Returns
    (Q, A11, A22, sigma_hat (numpy int8), p, info): Q^T Sigma Q = diag(sigma_hat) and
    Q^{-1} H Q = diag(A11, A22) with Q^{-1} = diag(sigma_hat) Q^T Sigma."""
    import numpy as np
    n, ldh = _check_H(H)
    h = _handle(handle)
    Q = torch.empty_like(H)
    A11 = torch.empty_like(H)
    A22 = torch.empty_like(H)
    keep, sp = _sigma(n, sigma)
    sh = np.zeros(n, dtype=np.int8)
    p = ctypes.c_int(0)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_gsplit(h._h, n, sp, ctypes.c_void_p(H.data_ptr()), ldh, ctypes.c_void_p(Q.data_ptr()),
                           Q.stride(0), ctypes.c_void_p(A11.data_ptr()), A11.stride(0),
                           ctypes.c_void_p(A22.data_ptr()), A22.stride(0), sh.ctypes.data_as(ctypes.c_void_p),
                           ctypes.byref(p), ctypes.byref(o), ctypes.byref(info))
    h._check(st)
    k = p.value
    return Q, A11[:k, :k], A22[:n - k, :n - k], sh, k, info.as_dict()


def sign_noalloc(H, S=None, sigma=None, handle=None, **kw):
    """pssd_sign_noalloc: S = sign(H) for n <= 128 with every temporary taken
    from the library's fixed device scratch array (no device allocation by the
    library; pass a preallocated S to allocate nothing at all).  Returns
    (S, info dict)."""
    n, ldh = _check_H(H)
    h = _handle(handle)
    if S is None:
        S = torch.empty_like(H)
    keep, sp = _sigma(n, sigma)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_sign_noalloc(h._h, n, sp, ctypes.c_void_p(H.data_ptr()), ldh, ctypes.c_void_p(S.data_ptr()),
                                 S.stride(0), ctypes.byref(o), ctypes.byref(info))
    h._check(st)
    return S, info.as_dict()


def split(H, sigma=None, handle=None, S=None, **kw):
    """One structure-preserving split.  S: optional precomputed sign(H) (an n x n
    row-major float64 CUDA tensor); None computes it.  Returns (Q, A11, A22, p, info)."""
    n, ldh = _check_H(H)
    h = _handle(handle)
    if S is not None:
        _check_H(S)
        if S.shape != H.shape:
            raise ValueError("S must match H")
    keep, sp = _sigma(n, sigma)
    p = int((keep > 0).sum()) if keep is not None else n // 2
    Q = torch.empty_like(H)
    A11 = torch.empty(max(p, 1), max(p, 1), dtype=H.dtype, device=H.device)
    A22 = torch.empty(max(n - p, 1), max(n - p, 1), dtype=H.dtype, device=H.device)
    pp = ctypes.c_int(0)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_split(h._h, n, sp, ctypes.c_void_p(H.data_ptr()), ldh,
                          ctypes.c_void_p(S.data_ptr() if S is not None else 0), S.stride(0) if S is not None else n,
                          ctypes.c_void_p(Q.data_ptr()), Q.stride(0), ctypes.c_void_p(A11.data_ptr()), A11.stride(0),
                          ctypes.c_void_p(A22.data_ptr()), A22.stride(0), ctypes.byref(pp), ctypes.byref(o),
                          ctypes.byref(info))
    h._check(st)
    return Q, A11[:p, :p], A22[:n - p, :n - p], pp.value, info.as_dict()


def eig(H, sigma=None, handle=None, **kw):
    """Full diagonalisation V^{-1} H V = diag(D).  Returns (D, V, info)."""
    n, ldh = _check_H(H)
    h = _handle(handle)
    keep, sp = _sigma(n, sigma)
    V = torch.empty_like(H)
    D = torch.empty(n, dtype=H.dtype, device=H.device)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_eig(h._h, n, sp, ctypes.c_void_p(H.data_ptr()), ldh, ctypes.c_void_p(V.data_ptr()),
                        V.stride(0), ctypes.c_void_p(D.data_ptr()), ctypes.byref(o), ctypes.byref(info))
    h._check(st)
    return D, V, info.as_dict()


def _check_block(X, k=None):
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float64 and X.dim() == 2
            and X.shape[0] == X.shape[1] and X.stride(1) == 1):
        raise ValueError("A and B must be square row-major float64 CUDA tensors")
    if k is not None and X.shape[0] != k:
        raise ValueError("A and B must have the same order")
    return X.shape[0], X.stride(0)


def casida_sign(A, B, handle=None, **kw):
    """sign(H) of the Casida matrix H = [[A, B], [-B, -A]] by the structure-aware
    k x k iteration (polar factor of C = L_P^T L_R).  Returns (S, info)."""
    k, lda = _check_block(A)
    _, ldb = _check_block(B, k)
    h = _handle(handle)
    S = torch.empty(2 * k, 2 * k, dtype=A.dtype, device=A.device)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_casida_sign(h._h, k, ctypes.c_void_p(A.data_ptr()), lda, ctypes.c_void_p(B.data_ptr()), ldb,
                                ctypes.c_void_p(S.data_ptr()), S.stride(0), ctypes.byref(o), ctypes.byref(info))
    h._check(st)
    return S, info.as_dict()


def casida_split(A, B, handle=None, **kw):
    """Structure-aware split of the Casida H.  Returns (Q, A11, A22, k, info)."""
    k, lda = _check_block(A)
    _, ldb = _check_block(B, k)
    h = _handle(handle)
    Q = torch.empty(2 * k, 2 * k, dtype=A.dtype, device=A.device)
    A11 = torch.empty(k, k, dtype=A.dtype, device=A.device)
    A22 = torch.empty(k, k, dtype=A.dtype, device=A.device)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_casida_split(h._h, k, ctypes.c_void_p(A.data_ptr()), lda, ctypes.c_void_p(B.data_ptr()), ldb,
                                 ctypes.c_void_p(Q.data_ptr()), Q.stride(0), ctypes.c_void_p(A11.data_ptr()),
                                 A11.stride(0), ctypes.c_void_p(A22.data_ptr()), A22.stride(0), ctypes.byref(o),
                                 ctypes.byref(info))
    h._check(st)
    return Q, A11, A22, k, info.as_dict()


def casida_eig(A, B, handle=None, **kw):
    """Structure-aware full diagonalisation of the Casida H.  Returns (D, V, info)."""
    k, lda = _check_block(A)
    _, ldb = _check_block(B, k)
    h = _handle(handle)
    V = torch.empty(2 * k, 2 * k, dtype=A.dtype, device=A.device)
    D = torch.empty(2 * k, dtype=A.dtype, device=A.device)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_casida_eig(h._h, k, ctypes.c_void_p(A.data_ptr()), lda, ctypes.c_void_p(B.data_ptr()), ldb,
                               ctypes.c_void_p(V.data_ptr()), V.stride(0), ctypes.c_void_p(D.data_ptr()),
                               ctypes.byref(o), ctypes.byref(info))
    h._check(st)
    return D, V, info.as_dict()


def sign_vjp(H, Sbar=None, lambar=None, sigma=None, handle=None, **kw):
    """dL/dH for L = <Sbar, sign(H)> + sum_i lambar_i lambda_i (eigenvalues in
    the output order of eig).  Sbar: n x n float64 CUDA tensor or None;
    lambar: length-n float64 CUDA tensor or None."""
    n, ldh = _check_H(H)
    h = _handle(handle)
    keep, sp = _sigma(n, sigma)
    if Sbar is not None:
        Sbar = Sbar.contiguous()
        if Sbar.shape != H.shape or Sbar.dtype != torch.float64 or not Sbar.is_cuda:
            raise ValueError("Sbar must match H")
    if lambar is not None:
        lambar = lambar.contiguous()
        if lambar.shape != (n,) or lambar.dtype != torch.float64 or not lambar.is_cuda:
            raise ValueError("lambar must be a length-n float64 CUDA tensor")
    Hbar = torch.empty_like(H)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_sign_vjp(h._h, n, sp, ctypes.c_void_p(H.data_ptr()), ldh,
                             ctypes.c_void_p(Sbar.data_ptr() if Sbar is not None else 0), n,
                             ctypes.c_void_p(lambar.data_ptr() if lambar is not None else 0),
                             ctypes.c_void_p(Hbar.data_ptr()), Hbar.stride(0), ctypes.byref(o), ctypes.byref(info))
    h._check(st)
    return Hbar


def sign_vjp_rev(H, Sbar=None, pos_weight=0.0, sigma=None, handle=None, **kw):
    """Step-reversal adjoint: dL/dH for L = <Sbar, sign(H)> + pos_weight * (sum of the
    positive eigenvalues), reversing each Zolotarev step through its recorded shifted
    inverses (flags=FLAG_RECOMPUTE: recompute them from per-step checkpoints).  The result
    is the gradient with respect to pseudosymmetric H."""
    n, ldh = _check_H(H)
    h = _handle(handle)
    keep, sp = _sigma(n, sigma)
    if Sbar is not None:
        Sbar = Sbar.contiguous()
        if Sbar.shape != H.shape or Sbar.dtype != torch.float64 or not Sbar.is_cuda:
            raise ValueError("Sbar must match H")
    Hbar = torch.empty_like(H)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_sign_vjp_rev(h._h, n, sp, ctypes.c_void_p(H.data_ptr()), ldh,
                                 ctypes.c_void_p(Sbar.data_ptr() if Sbar is not None else 0), n,
                                 ctypes.c_double(pos_weight), ctypes.c_void_p(Hbar.data_ptr()), Hbar.stride(0),
                                 ctypes.byref(o), ctypes.byref(info))
    h._check(st)
    return Hbar


def _check_Hz(H):
    if not (isinstance(H, torch.Tensor) and H.is_cuda and H.dtype == torch.complex128 and H.dim() == 2
            and H.shape[0] == H.shape[1] and H.stride(1) == 1):
        raise ValueError("H must be a square row-major complex128 CUDA tensor")
    return H.shape[0], H.stride(0)


def zsign(H, sigma=None, handle=None, **kw):
    """sign(H) of a complex pseudo-Hermitian H (complex128 CUDA tensor; the BSE forms).
    Returns (S, info)."""
    n, ldh = _check_Hz(H)
    h = _handle(handle)
    keep, sp = _sigma(n, sigma)
    S = torch.empty_like(H)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_zsign(h._h, n, sp, ctypes.c_void_p(H.data_ptr()), ldh, ctypes.c_void_p(S.data_ptr()),
                          S.stride(0), ctypes.byref(o), ctypes.byref(info))
    h._check(st)
    return S, info.as_dict()


def zeig(H, sigma=None, handle=None, **kw):
    """Full diagonalisation of a complex pseudo-Hermitian H: (D real, V complex, info) with
    V^{-1} H V = diag(D) and V^H Sigma V = diag(sign(D))."""
    n, ldh = _check_Hz(H)
    h = _handle(handle)
    keep, sp = _sigma(n, sigma)
    V = torch.empty_like(H)
    D = torch.empty(n, dtype=torch.float64, device=H.device)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_zeig(h._h, n, sp, ctypes.c_void_p(H.data_ptr()), ldh, ctypes.c_void_p(V.data_ptr()),
                         V.stride(0), ctypes.c_void_p(D.data_ptr()), ctypes.byref(o), ctypes.byref(info))
    h._check(st)
    return D, V, info.as_dict()


class SignFn(torch.autograd.Function):
    """S = sign(H) with the library's adjoint as backward (FP64).  adjoint="steps" (default)
    reverses the Zolotarev steps (gradient with respect to pseudosymmetric H); "spectral"
    uses the Daleckii-Krein form on the eigendecomposition (unconstrained gradient)."""

    @staticmethod
    def forward(ctx, H, sigma=None, adjoint="steps"):
        S, _ = sign(H.detach(), sigma=sigma)
        ctx.save_for_backward(H)
        ctx.sigma = sigma
        ctx.adjoint = adjoint
        return S

    @staticmethod
    def backward(ctx, gS):
        (H,) = ctx.saved_tensors
        if ctx.adjoint == "steps":
            return sign_vjp_rev(H.detach(), Sbar=gS.contiguous(), sigma=ctx.sigma), None, None
        return sign_vjp(H.detach(), Sbar=gS.contiguous(), sigma=ctx.sigma), None, None


class EigvalsFn(torch.autograd.Function):
    """Eigenvalues of H (output order of eig) with the library's adjoint as backward."""

    @staticmethod
    def forward(ctx, H, sigma=None):
        D, _, _ = eig(H.detach(), sigma=sigma)
        ctx.save_for_backward(H)
        ctx.sigma = sigma
        return D

    @staticmethod
    def backward(ctx, gD):
        (H,) = ctx.saved_tensors
        return sign_vjp(H.detach(), lambar=gD.contiguous(), sigma=ctx.sigma), None


def eig_batched(Hs, sigmas=None, handle=None, **kw):
    """Full diagonalisation of a list of square float64 CUDA tensors of any
    orders in one call.  Returns (list of D, list of V, list of info dicts)."""
    count = len(Hs)
    h = _handle(handle)
    ns = (ctypes.c_int * count)(); lds = (ctypes.c_int * count)(); ldv = (ctypes.c_int * count)()
    Hp = (ctypes.c_void_p * count)(); Vp = (ctypes.c_void_p * count)(); Dp = (ctypes.c_void_p * count)()
    Vs, Ds, keep = [], [], []
    sp = None
    if sigmas is not None:
        sp = (ctypes.c_void_p * count)()
    for i, H in enumerate(Hs):
        n, ld = _check_H(H)
        V = torch.empty_like(H); D = torch.empty(n, dtype=H.dtype, device=H.device)
        ns[i] = n; lds[i] = ld; ldv[i] = V.stride(0)
        Hp[i] = H.data_ptr(); Vp[i] = V.data_ptr(); Dp[i] = D.data_ptr()
        Vs.append(V); Ds.append(D)
        if sigmas is not None:
            k, ptr = _sigma(n, sigmas[i])
            keep.append(k)
            sp[i] = ptr.value if ptr is not None else None
    infos = (Info * count)()
    o = _opts(**kw)
    st = lib().pssd_eig_batched(h._h, count, ns, sp, Hp, lds, Vp, ldv, Dp, ctypes.byref(o), infos)
    h._check(st)
    return Ds, Vs, [infos[i].as_dict() for i in range(count)]


def test_sym_eig(B, handle=None, **kw):
    """Test hook: the symmetric divide-and-conquer (Alg. 2) on a symmetric float64
    CUDA tensor B.  Returns (w, W, info), eigenvalues unordered."""
    m, ldb = _check_H(B)
    h = _handle(handle)
    W = torch.empty_like(B)
    w = torch.empty(m, dtype=B.dtype, device=B.device)
    info = Info()
    o = _opts(**kw)
    st = lib().pssd_test_sym_eig(h._h, m, ctypes.c_void_p(B.data_ptr()), ldb, ctypes.c_void_p(W.data_ptr()),
                                 W.stride(0), ctypes.c_void_p(w.data_ptr()), ctypes.byref(o), ctypes.byref(info))
    h._check(st)
    return w, W, info.as_dict()


def test_krylov(A, op=0, steps=24, power=0, seed=1, fused=True, want_v0=True, handle=None):
    """Test hook: the library's Krylov loops on a float64 CUDA matrix A (op 0: A x with A
    symmetric; op 1: A^T (A x) with A lower triangular), step by step or in one cluster
    launch.  Returns (out, v0): Lanczos alphas/betas (2 steps + 2 entries: alpha_j at j,
    beta_j at steps + 1 + j) or [v^T op(A) v] after `power` power steps, and the
    starting vector before normalisation (None unless want_v0)."""
    m, lda = _check_H(A)
    h = _handle(handle)
    out = torch.zeros(2 * steps + 2 if power == 0 else 1, dtype=torch.float64, device=A.device)
    v0 = torch.empty(m, dtype=torch.float64, device=A.device) if want_v0 else None
    st = lib().pssd_test_krylov(h._h, op, m, ctypes.c_void_p(A.data_ptr()), lda, steps, power, seed,
                                1 if fused else 0, ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(v0.data_ptr() if v0 is not None else None))
    h._check(st)
    return out, v0


def test_gemm_f32(A, B, use_tc=True, ta=0, tb=0, triA=0, triB=0, lowerC=0, alpha=1.0, beta=0.0, Cin=None,
                  kscale=None, handle=None):
    """Test hook: C = alpha op(A) diag(kscale) op(B) + beta Cin with the library's FP32 GEMM
    (tensor cores or SIMT).  A, B: float32 CUDA tensors, 2-D or 3-D (batch first)."""
    h = _handle(handle)
    batched = A.dim() == 3
    A3 = A if batched else A[None]; B3 = B if batched else B[None]
    nb = A3.shape[0]
    m = A3.shape[2] if ta else A3.shape[1]; k = A3.shape[1] if ta else A3.shape[2]
    n = B3.shape[1] if tb else B3.shape[2]
    C = torch.empty(nb, m, n, dtype=torch.float32, device=A.device)
    if Cin is None:
        Cin3 = C
    else:
        Cin3 = Cin if Cin.dim() == 3 else Cin[None]
    st = lib().pssd_test_gemm_f32(h._h, 1 if use_tc else 0, m, n, k, nb, ta, tb, triA, triB, lowerC,
                                  float(alpha), float(beta),
                                  ctypes.c_void_p(A3.data_ptr()), A3.stride(1), A3.stride(0) if nb > 1 else 0,
                                  ctypes.c_void_p(B3.data_ptr()), B3.stride(1), B3.stride(0) if nb > 1 else 0,
                                  ctypes.c_void_p(Cin3.data_ptr()), Cin3.stride(1), Cin3.stride(0) if nb > 1 else 0,
                                  ctypes.c_void_p(C.data_ptr()), C.stride(1), C.stride(0),
                                  ctypes.c_void_p(kscale.data_ptr() if kscale is not None else 0))
    h._check(st)
    return C if batched else C[0]


def test_gemm_f64(A, B, engine=2, ta=0, tb=0, triA=0, triB=0, lowerC=0, alpha=1.0, beta=0.0, Cin=None,
                  kscale=None, handle=None):
    """Test hook: the FP64 contraction with engine 0 (DFMA), 1 (float pairs) or 2 (tensor-core slices)."""
    h = _handle(handle)
    batched = A.dim() == 3
    A3 = A if batched else A[None]; B3 = B if batched else B[None]
    nb = A3.shape[0]
    m = A3.shape[2] if ta else A3.shape[1]; k = A3.shape[1] if ta else A3.shape[2]
    n = B3.shape[1] if tb else B3.shape[2]
    C = torch.empty(nb, m, n, dtype=torch.float64, device=A.device)
    Cin3 = C if Cin is None else (Cin if Cin.dim() == 3 else Cin[None])
    st = lib().pssd_test_gemm_f64(h._h, int(engine), m, n, k, nb, ta, tb, triA, triB, lowerC,
                                  float(alpha), float(beta),
                                  ctypes.c_void_p(A3.data_ptr()), A3.stride(1), A3.stride(0) if nb > 1 else 0,
                                  ctypes.c_void_p(B3.data_ptr()), B3.stride(1), B3.stride(0) if nb > 1 else 0,
                                  ctypes.c_void_p(Cin3.data_ptr()), Cin3.stride(1), Cin3.stride(0) if nb > 1 else 0,
                                  ctypes.c_void_p(C.data_ptr()), C.stride(1), C.stride(0),
                                  ctypes.c_void_p(kscale.data_ptr() if kscale is not None else 0))
    h._check(st)
    return C if batched else C[0]
