"""Thin Python binding of libloopnest (the C ABI in include/loopnest.h).

Argument marshalling only: every step of every operation runs in the CUDA
kernels of libloopnest.so. PyTorch provides device memory (tensors and the
workspace) and the current CUDA stream. There is no CPU fallback: if the
shared library has not been built, every call raises.

Names follow the C ABI (ln_gemm -> gemm, ...). `form` is "plain" or
"internalized"; `prec` is "fp32", "bf16", "3xbf16", "6xbf16", "tf32" or "3xtf32".
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libloopnest.so")

FORMS = {"plain": 0, "internalized": 1}
PRECS = {"fp32": 0, "bf16": 1, "3xbf16": 2, "6xbf16": 3, "tf32": 4, "3xtf32": 5}
FILLS = {"full": 0, "lower": 1, "upper": 2}
# MMA products per multiply-add of each precision (for effective-peak accounting)
PRODUCTS = {"fp32": 1, "bf16": 1, "3xbf16": 3, "6xbf16": 6, "tf32": 1, "3xtf32": 3}

STATUS = {
    0: "LN_SUCCESS", 1: "LN_ERR_INVALID_VALUE", 2: "LN_ERR_ALIASING", 3: "LN_ERR_MISALIGNED",
    4: "LN_ERR_UNSUPPORTED", 5: "LN_ERR_CUDA", 6: "LN_ERR_TIMEOUT", 7: "LN_ERR_WORKSPACE",
}


class LoopnestError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")


class SymDesc(ctypes.Structure):
    """ln_sym_desc"""
    _fields_ = [
        ("n", ctypes.c_int), ("k", ctypes.c_int),
        ("A", ctypes.c_void_p), ("lda", ctypes.c_int),
        ("B", ctypes.c_void_p), ("ldb", ctypes.c_int),
        ("C", ctypes.c_void_p), ("ldc", ctypes.c_int),
    ]


_lib = None

_I, _F, _P, _SZ = ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t
_SIGS = {
    "ln_get_last_error": (ctypes.c_char_p, []),
    "ln_status_string": (ctypes.c_char_p, [_I]),
    "ln_version": (_I, []),
    "ln_stream_check": (_I, [_P]),
    "ln_launch_count": (ctypes.c_longlong, []),
    "ln_timing_enable": (_I, [_I]),
    "ln_timing_read": (_I, [ctypes.c_char_p, _P, _P]),
    "ln_peak_probe": (_I, [_I, ctypes.c_longlong, _P, _P, ctypes.c_longlong, _P, _P]),
    "ln_set_tuning": (_I, [ctypes.c_char_p, _I]),
    "ln_get_tuning": (_I, [ctypes.c_char_p, _P]),
    "ln_gemm_workspace_size": (_I, [_I, _I, _I, _I, _I, _P]),
    "ln_gemm": (_I, [_I, _I, _I, _F, _P, _I, _P, _I, _F, _P, _I, _P, _SZ, _I, _I, _P]),
    "ln_gemm_chain_workspace_size": (_I, [_I, _I, _I, _I, _I, _I, _P]),
    "ln_gemm_chain": (_I, [_I, _I, _I, _I, _F, _P, _P, _P, _F, _P, _P, _P, _P, _SZ, _I, _I, _P]),
    "ln_3mm_workspace_size": (_I, [_I, _I, _I, _I, _I, _I, _I, _P]),
    "ln_3mm": (_I, [_I, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _SZ, _I, _I, _P]),
    "ln_3mm_bwd_workspace_size": (_I, [_I, _I, _I, _I, _I, _I, _I, _P]),
    "ln_3mm_bwd": (_I, [_I, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _I, _I, _P]),
    "ln_col_stats_workspace_size": (_I, [_I, _I, _I, _P]),
    "ln_col_stats": (_I, [_I, _I, _P, _I, _P, _P, _P, _SZ, _I, _P]),
    "ln_gramschmidt": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _I, _P]),
    "ln_covariance_workspace_size": (_I, [_I, _I, _I, _I, _P]),
    "ln_covariance": (_I, [_I, _I, _P, _I, _P, _I, _P, _SZ, _I, _I, _P]),
    "ln_correlation": (_I, [_I, _I, _P, _I, _P, _I, _P, _SZ, _I, _I, _P]),
    "ln_covariance_fwd": (_I, [_I, _I, _P, _I, _P, _I, _P, _P, _SZ, _I, _I, _P]),
    "ln_correlation_fwd": (_I, [_I, _I, _P, _I, _P, _I, _P, _P, _SZ, _I, _I, _P]),
    "ln_covariance_noalloc": (_I, [_I, _I, _P, _I, _P, _I, _P]),
    "ln_syrk_workspace_size": (_I, [_I, _I, _I, _I, _P]),
    "ln_syrk": (_I, [_I, _I, _I, _F, _P, _I, _F, _P, _I, _P, _SZ, _I, _I, _P]),
    "ln_syr2k_workspace_size": (_I, [_I, _I, _I, _I, _P]),
    "ln_syr2k": (_I, [_I, _I, _I, _F, _P, _I, _P, _I, _F, _P, _I, _P, _SZ, _I, _I, _P]),
    "ln_syrk_batched_workspace_size": (_I, [_I, _P, _I, _I, _P]),
    "ln_syrk_batched": (_I, [_I, _I, _P, _P, _F, _F, _P, _SZ, _I, _I, _P]),
    "ln_syr2k_batched_workspace_size": (_I, [_I, _P, _I, _I, _P]),
    "ln_syr2k_batched": (_I, [_I, _I, _P, _P, _F, _F, _P, _SZ, _I, _I, _P]),
    "ln_gemm_chain_bwd_workspace_size": (_I, [_I, _I, _I, _I, _I, _I, _P]),
    "ln_gemm_chain_bwd": (_I, [_I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _I, _I, _P]),
    "ln_covariance_bwd_workspace_size": (_I, [_I, _I, _I, _I, _P]),
    "ln_covariance_bwd": (_I, [_I, _I, _P, _I, _P, _I, _P, _P, _I, _P, _SZ, _I, _I, _P]),
    "ln_correlation_bwd": (_I, [_I, _I, _P, _I, _P, _I, _P, _P, _I, _P, _SZ, _I, _I, _P]),
}
EXPORTS = tuple(_SIGS)


def lib():
    """The loaded libloopnest (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libloopnest.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != 0:
        msg = lib().ln_get_last_error().decode(errors="replace")
        raise LoopnestError(status, where, msg)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _enum(table, v, what):
    if isinstance(v, int):
        return v
    try:
        return table[v.lower()]
    except KeyError:
        raise ValueError(f"unknown {what} {v!r}; expected one of {sorted(table)}") from None


def _f32(t, name, host_ok=False):
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a float32 tensor")
    if not t.is_cuda and not (host_ok and t.is_pinned()):
        raise TypeError(f"{name} must be a CUDA tensor" + (" or a pinned host tensor" if host_ok else ""))
    if t.dim() != 2 or (t.stride(1) != 1 and t.numel() > 0):
        raise ValueError(f"{name} must be a 2-D row-major tensor (unit column stride)")
    return t


def _ld(t):
    return max(t.stride(0), t.shape[1]) if t.shape[0] > 1 else t.shape[1]


def _ws_query(fn, *args):
    n = ctypes.c_size_t(0)
    _check(getattr(lib(), fn)(*args, ctypes.byref(n)), fn)
    return int(n.value)


def _autotune(op, shape, prec):
    if os.environ.get("LN_AUTOTUNE", "off").lower() in ("cached", "search"):
        from . import autotune

        autotune.apply(op, shape, prec if isinstance(prec, str) else
                       {v: k for k, v in PRECS.items()}.get(prec, "fp32"))


def _workspace(nbytes, device):
    if nbytes == 0:
        return None, 0
    return torch.empty(nbytes, dtype=torch.uint8, device=device), nbytes


def launch_count() -> int:
    """Kernels libloopnest has launched in this process."""
    return int(lib().ln_launch_count())


def timing_enable(on=True) -> None:
    """Bracket library kernel launches with CUDA events on their streams: False
    or 0 off, True or 1 one event pair per launch, 2 spans (back-to-back
    launches with programmatic overlap share one pair; see loopnest.h)."""
    _check(lib().ln_timing_enable(int(on)), "ln_timing_enable")


def timing_read(family: str):
    """(total_ms, launches) of one kernel family since the last read."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int(0)
    _check(lib().ln_timing_read(family.encode(), ctypes.byref(ms), ctypes.byref(n)), "ln_timing_read")
    return float(ms.value), int(n.value)


def set_tuning(key: str, value: int) -> None:
    """Set a process-wide knob: "chunk_kt", "tile_n", "pack_threads", "split_k", "stream_k", "pair",
    "stage_beta", "stage_out", "sym_wide" (tensor-core engine), "simt_exact", "simt_tile" (FP32 tiled form) or "gs_rows"
    (Gram-Schmidt panel); the values each takes are listed in loopnest.h."""
    _check(lib().ln_set_tuning(key.encode(), int(value)), "ln_set_tuning")


def get_tuning(key: str) -> int:
    v = ctypes.c_int(0)
    _check(lib().ln_get_tuning(key.encode(), ctypes.byref(v)), "ln_get_tuning")
    return int(v.value)


PEAK_KINDS = {"mma_bf16": 0, "mma_tf32": 1, "ffma": 2, "copy": 3}


def peak_probe(kind, iters=1, src=None, dst=None, stream=None) -> float:
    """Launch one peak probe ("mma_bf16", "mma_tf32", "ffma" or "copy"; see
    ln_peak_probe in loopnest.h) on the stream and return its algorithmic work
    (flops, or bytes read plus written). `dst` is the probe's error word or
    sink (MMA, FFMA) or the copy's destination; `src` the copy's source."""
    work = ctypes.c_double(0.0)
    nbytes = 0 if dst is None else dst.numel() * dst.element_size()
    if src is not None and src.numel() * src.element_size() < nbytes:
        raise ValueError("the copy probe's source is smaller than its destination")
    _check(lib().ln_peak_probe(_enum(PEAK_KINDS, kind, "probe"), int(iters), _ptr(src), _ptr(dst), nbytes,
                               ctypes.byref(work), _stream(stream)), "ln_peak_probe")
    return float(work.value)


def stream_check(stream=None):
    """Synchronise the stream and raise if a kernel gave up a bounded wait."""
    _check(lib().ln_stream_check(_stream(stream)), "ln_stream_check")


# ---------------------------------------------------------------- forward operations
def gemm(A, B, C, alpha=1.0, beta=0.0, form="internalized", prec="3xbf16", stream=None):
    """C = alpha*A@B + beta*C in place; returns C."""
    _f32(A, "A"), _f32(B, "B"), _f32(C, "C")
    M, K = A.shape
    K2, N = B.shape
    if K2 != K or tuple(C.shape) != (M, N):
        raise ValueError("shape mismatch")
    fm, pr = _enum(FORMS, form, "form"), _enum(PRECS, prec, "precision")
    _autotune("gemm", (M, N, K), prec)
    ws, nb = _workspace(_ws_query("ln_gemm_workspace_size", M, N, K, fm, pr), A.device)
    _check(lib().ln_gemm(M, N, K, alpha, _ptr(A), _ld(A), _ptr(B), _ld(B), beta, _ptr(C), _ld(C), _ptr(ws), nb,
                         fm, pr, _stream(stream)), "ln_gemm")
    return C


def gemm_chain(A, B, C, D=None, alpha=1.0, beta=0.0, form="internalized", prec="3xbf16", stream=None, out=None):
    """E = (A@B)@C, F = alpha*E + beta*D. Returns (E, F).

    Operands and outputs may be pinned host tensors: the kernels then read and
    write them in host memory directly (no staging copies); new outputs follow
    A's placement. The workspace is always on the current GPU."""
    for t, nme in ((A, "A"), (B, "B"), (C, "C")):
        _f32(t, nme, host_ok=True)
        if not t.is_contiguous():
            raise ValueError(f"{nme} must be contiguous")
    ni, nk = A.shape
    nj, nl = B.shape[1], C.shape[1]
    if B.shape[0] != nk or C.shape[0] != nj:
        raise ValueError("shape mismatch")
    if D is not None:
        _f32(D, "D", host_ok=True)
        if tuple(D.shape) != (ni, nl) or not D.is_contiguous():
            raise ValueError("D must be contiguous ni x nl")
    fm, pr = _enum(FORMS, form, "form"), _enum(PRECS, prec, "precision")
    if out is None:
        pin = not A.is_cuda
        E = torch.empty((ni, nl), dtype=torch.float32, device=A.device, pin_memory=pin)
        F = torch.empty((ni, nl), dtype=torch.float32, device=A.device, pin_memory=pin)
    else:
        E, F = out
        _f32(E, "E", host_ok=True), _f32(F, "F", host_ok=True)
    dev = A.device if A.is_cuda else torch.device("cuda", torch.cuda.current_device())
    _autotune("gemm_chain", (ni, nj, nk, nl), prec)
    ws, nb = _workspace(_ws_query("ln_gemm_chain_workspace_size", ni, nj, nk, nl, fm, pr), dev)
    _check(lib().ln_gemm_chain(ni, nj, nk, nl, alpha, _ptr(A), _ptr(B), _ptr(C), beta, _ptr(D), _ptr(E), _ptr(F),
                               _ptr(ws), nb, fm, pr, _stream(stream)), "ln_gemm_chain")
    return E, F


def three_mm(A, B, C, D, form="internalized", prec="3xbf16", stream=None, out=None):
    """G = (A@B)@(C@D) (polybench 3mm); returns G. Operands may be pinned host
    tensors as for gemm_chain."""
    for t, nme in ((A, "A"), (B, "B"), (C, "C"), (D, "D")):
        _f32(t, nme, host_ok=True)
        if not t.is_contiguous():
            raise ValueError(f"{nme} must be contiguous")
    ni, nk = A.shape
    nj, nm, nl = B.shape[1], C.shape[1], D.shape[1]
    if B.shape[0] != nk or C.shape[0] != nj or D.shape[0] != nm:
        raise ValueError("shape mismatch")
    fm, pr = _enum(FORMS, form, "form"), _enum(PRECS, prec, "precision")
    if out is None:
        G = torch.empty((ni, nl), dtype=torch.float32, device=A.device, pin_memory=not A.is_cuda)
    else:
        G = out
        _f32(G, "G", host_ok=True)
        if tuple(G.shape) != (ni, nl) or not G.is_contiguous():
            raise ValueError("out must be contiguous ni x nl")
    dev = A.device if A.is_cuda else torch.device("cuda", torch.cuda.current_device())
    _autotune("three_mm", (ni, nj, nk, nl, nm), prec)
    ws, nb = _workspace(_ws_query("ln_3mm_workspace_size", ni, nj, nk, nl, nm, fm, pr), dev)
    _check(lib().ln_3mm(ni, nj, nk, nl, nm, _ptr(A), _ptr(B), _ptr(C), _ptr(D), _ptr(G), _ptr(ws), nb, fm, pr,
                        _stream(stream)), "ln_3mm")
    return G


def gramschmidt(A, form="internalized", stream=None, Q=None, R=None, in_place=False):
    """(Q, R) of modified Gram-Schmidt on A (m x n, polybench gramschmidt).

    With in_place=True, A is overwritten by Q (the benchmark's semantics) and
    returned as Q. Q and R may be given as preallocated outputs."""
    _f32(A, "A")
    m, n = A.shape
    fm = _enum(FORMS, form, "form")
    if in_place:
        Q = A
    elif Q is None:
        Q = torch.empty((m, n), dtype=torch.float32, device=A.device)
    else:
        _f32(Q, "Q")
        if tuple(Q.shape) != (m, n):
            raise ValueError("Q must be m x n")
    if R is None:
        R = torch.empty((n, n), dtype=torch.float32, device=A.device)
    else:
        _f32(R, "R")
        if tuple(R.shape) != (n, n):
            raise ValueError("R must be n x n")
    _check(lib().ln_gramschmidt(m, n, _ptr(A), _ld(A), _ptr(Q), _ld(Q), _ptr(R), _ld(R), fm, _stream(stream)),
           "ln_gramschmidt")
    return Q, R


def col_stats(X, form="internalized", stream=None):
    """(mean, ss) of the columns of X, float64."""
    _f32(X, "X")
    n, m = X.shape
    fm = _enum(FORMS, form, "form")
    mean = torch.empty(m, dtype=torch.float64, device=X.device)
    ss = torch.empty(m, dtype=torch.float64, device=X.device)
    ws, nb = _workspace(_ws_query("ln_col_stats_workspace_size", n, m, fm), X.device)
    _check(lib().ln_col_stats(n, m, _ptr(X), _ld(X), _ptr(mean), _ptr(ss), _ptr(ws), nb, fm, _stream(stream)),
           "ln_col_stats")
    return mean, ss


def _covlike(fn, X, form, prec, stream, out, stats=None):
    _f32(X, "X")
    n, m = X.shape
    fm, pr = _enum(FORMS, form, "form"), _enum(PRECS, prec, "precision")
    out = torch.empty((m, m), dtype=torch.float32, device=X.device) if out is None else out
    _autotune("covariance" if fn.startswith("ln_covariance") else "correlation", (n, m), prec)
    ws, nb = _workspace(_ws_query("ln_covariance_workspace_size", n, m, fm, pr), X.device)
    if stats is None:
        _check(getattr(lib(), fn)(n, m, _ptr(X), _ld(X), _ptr(out), _ld(out), _ptr(ws), nb, fm, pr, _stream(stream)),
               fn)
    else:
        _check(getattr(lib(), fn)(n, m, _ptr(X), _ld(X), _ptr(out), _ld(out), _ptr(stats), _ptr(ws), nb, fm, pr,
                                  _stream(stream)), fn)
    return out


def covariance(X, form="internalized", prec="3xbf16", stream=None, out=None):
    return _covlike("ln_covariance", X, form, prec, stream, out)


def correlation(X, form="internalized", prec="3xbf16", stream=None, out=None):
    return _covlike("ln_correlation", X, form, prec, stream, out)


def covariance_fwd(X, form="internalized", prec="3xbf16", stream=None, out=None):
    """(cov, stats): the covariance and the FP64 [mean; ss] (2*nfeat) that
    covariance_bwd takes, from one call."""
    stats = torch.empty(2 * X.shape[1], dtype=torch.float64, device=X.device)
    return _covlike("ln_covariance_fwd", X, form, prec, stream, out, stats), stats


def correlation_fwd(X, form="internalized", prec="3xbf16", stream=None, out=None):
    """(corr, stats): the correlation and the FP64 [mean; ss] (2*nfeat) that
    correlation_bwd takes, from one call."""
    stats = torch.empty(2 * X.shape[1], dtype=torch.float64, device=X.device)
    return _covlike("ln_correlation_fwd", X, form, prec, stream, out, stats), stats


def syrk(A, C, alpha=1.0, beta=0.0, fill="full", form="internalized", prec="3xbf16", stream=None):
    """C = alpha*A@A.T + beta*C on `fill`, in place; returns C."""
    _f32(A, "A"), _f32(C, "C")
    n, k = A.shape
    fm, pr, fl = _enum(FORMS, form, "form"), _enum(PRECS, prec, "precision"), _enum(FILLS, fill, "fill")
    _autotune("syrk", (n, k), prec)
    ws, nb = _workspace(_ws_query("ln_syrk_workspace_size", n, k, fm, pr), A.device)
    _check(lib().ln_syrk(fl, n, k, alpha, _ptr(A), _ld(A), beta, _ptr(C), _ld(C), _ptr(ws), nb, fm, pr,
                         _stream(stream)), "ln_syrk")
    return C


def syr2k(A, B, C, alpha=1.0, beta=0.0, fill="full", form="internalized", prec="3xbf16", stream=None):
    """C = alpha*(A@B.T + B@A.T) + beta*C on `fill`, in place; returns C."""
    _f32(A, "A"), _f32(B, "B"), _f32(C, "C")
    n, k = A.shape
    fm, pr, fl = _enum(FORMS, form, "form"), _enum(PRECS, prec, "precision"), _enum(FILLS, fill, "fill")
    _autotune("syr2k", (n, k), prec)
    ws, nb = _workspace(_ws_query("ln_syr2k_workspace_size", n, k, fm, pr), A.device)
    _check(lib().ln_syr2k(fl, n, k, alpha, _ptr(A), _ld(A), _ptr(B), _ld(B), beta, _ptr(C), _ld(C), _ptr(ws), nb, fm,
                          pr, _stream(stream)), "ln_syr2k")
    return C


class SymBatch:
    """A batched SYRK/SYR2K call over lists of tensors of uneven sizes.

    Construction validates the instances, builds the host and device
    descriptor arrays and sizes the workspace; ``run()`` then only launches
    kernels, so it may be captured in a CUDA graph and replayed.
    """

    def __init__(self, As, Cs, Bs=None, alpha=1.0, beta=0.0, fill="full", form="internalized", prec="3xbf16"):
        self.two = Bs is not None
        self.count = len(As)
        self.alpha, self.beta = float(alpha), float(beta)
        self.fill = _enum(FILLS, fill, "fill")
        self.form, self.prec = _enum(FORMS, form, "form"), _enum(PRECS, prec, "precision")
        self.tensors = (list(As), list(Cs), list(Bs) if Bs is not None else None)
        arr = (SymDesc * max(self.count, 1))()
        for i, A in enumerate(As):
            _f32(A, "A"), _f32(Cs[i], "C")
            B = Bs[i] if Bs is not None else None
            if B is not None:
                _f32(B, "B")
            arr[i] = SymDesc(A.shape[0], A.shape[1], A.data_ptr(), _ld(A), B.data_ptr() if B is not None else None,
                             _ld(B) if B is not None else 0, Cs[i].data_ptr(), _ld(Cs[i]))
        self.h_descs = arr
        dev = As[0].device if self.count else torch.device("cuda")
        raw = bytes(memoryview(arr).cast("B"))
        self.d_descs = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(dev)
        pre = "ln_syr2k" if self.two else "ln_syrk"
        self.fn = pre + "_batched"
        nb = _ws_query(pre + "_batched_workspace_size", self.count, ctypes.byref(arr), self.form, self.prec)
        self.ws, self.nb = _workspace(nb, dev)

    def run(self, stream=None):
        if self.count:
            # the batch's class for the autotuner: count and mean instance sizes
            ns = [d.n for d in self.h_descs[:self.count]]
            ks = [d.k for d in self.h_descs[:self.count]]
            _autotune(self.fn[3:], (self.count, sum(ns) // self.count, max(sum(ks) // self.count, 1)), self.prec)
        _check(getattr(lib(), self.fn)(self.fill, self.count, ctypes.byref(self.h_descs), _ptr(self.d_descs),
                                       self.alpha, self.beta, _ptr(self.ws), self.nb, self.form, self.prec,
                                       _stream(stream)), self.fn)


# ---------------------------------------------------------------- adjoints
def gemm_chain_bwd(A, B, C, G, form="internalized", prec="3xbf16", stream=None):
    """(dA, dB, dC) for E = (A@B)@C with upstream gradient G."""
    for t, nme in ((A, "A"), (B, "B"), (C, "C"), (G, "G")):
        _f32(t, nme)
        if not t.is_contiguous():
            raise ValueError(f"{nme} must be contiguous")
    ni, nk = A.shape
    nj, nl = B.shape[1], C.shape[1]
    fm, pr = _enum(FORMS, form, "form"), _enum(PRECS, prec, "precision")
    dA, dB, dC = torch.empty_like(A), torch.empty_like(B), torch.empty_like(C)
    ws, nb = _workspace(_ws_query("ln_gemm_chain_bwd_workspace_size", ni, nj, nk, nl, fm, pr), A.device)
    _check(lib().ln_gemm_chain_bwd(ni, nj, nk, nl, _ptr(A), _ptr(B), _ptr(C), _ptr(G), _ptr(dA), _ptr(dB), _ptr(dC),
                                   _ptr(ws), nb, fm, pr, _stream(stream)), "ln_gemm_chain_bwd")
    return dA, dB, dC


def _cov_bwd(fn, X, W, stats, form, prec, stream):
    _f32(X, "X"), _f32(W, "W")
    n, m = X.shape
    fm, pr = _enum(FORMS, form, "form"), _enum(PRECS, prec, "precision")
    dX = torch.empty((n, m), dtype=torch.float32, device=X.device)
    ws, nb = _workspace(_ws_query("ln_covariance_bwd_workspace_size", n, m, fm, pr), X.device)
    _check(getattr(lib(), fn)(n, m, _ptr(X), _ld(X), _ptr(W), _ld(W), _ptr(stats), _ptr(dX), m, _ptr(ws), nb, fm, pr,
                              _stream(stream)), fn)
    return dX


def covariance_bwd(X, W, stats=None, form="internalized", prec="3xbf16", stream=None):
    return _cov_bwd("ln_covariance_bwd", X, W, stats, form, prec, stream)


def correlation_bwd(X, W, stats=None, form="internalized", prec="3xbf16", stream=None):
    return _cov_bwd("ln_correlation_bwd", X, W, stats, form, prec, stream)


def three_mm_bwd(A, B, C, D, Gb, form="internalized", prec="3xbf16", stream=None):
    """(dA, dB, dC, dD) for G = (A@B)@(C@D) with upstream gradient Gb."""
    for t, nme in ((A, "A"), (B, "B"), (C, "C"), (D, "D"), (Gb, "Gb")):
        _f32(t, nme)
        if not t.is_contiguous():
            raise ValueError(f"{nme} must be contiguous")
    ni, nk = A.shape
    nj, nm, nl = B.shape[1], C.shape[1], D.shape[1]
    if B.shape[0] != nk or C.shape[0] != nj or D.shape[0] != nm or tuple(Gb.shape) != (ni, nl):
        raise ValueError("shape mismatch")
    fm, pr = _enum(FORMS, form, "form"), _enum(PRECS, prec, "precision")
    grads = [torch.empty(x.shape, dtype=torch.float32, device=A.device) for x in (A, B, C, D)]
    ws, nb = _workspace(_ws_query("ln_3mm_bwd_workspace_size", ni, nj, nk, nl, nm, fm, pr), A.device)
    _check(lib().ln_3mm_bwd(ni, nj, nk, nl, nm, _ptr(A), _ptr(B), _ptr(C), _ptr(D), _ptr(Gb),
                            *(_ptr(g) for g in grads), _ptr(ws), nb, fm, pr, _stream(stream)), "ln_3mm_bwd")
    return tuple(grads)


class ThreeMmFn(torch.autograd.Function):
    """G = (A@B)@(C@D) with the hand-written adjoint (ln_3mm_bwd)."""

    @staticmethod
    def forward(ctx, A, B, C, D, form="internalized", prec="3xbf16"):
        ts = [t.contiguous() for t in (A, B, C, D)]
        ctx.save_for_backward(*ts)
        ctx.cfg = (form, prec)
        return three_mm(*ts, form=form, prec=prec)

    @staticmethod
    def backward(ctx, gG):
        A, B, C, D = ctx.saved_tensors
        dA, dB, dC, dD = three_mm_bwd(A, B, C, D, gG.contiguous(), *ctx.cfg)
        return dA, dB, dC, dD, None, None


class GemmChainFn(torch.autograd.Function):
    """E = (A@B)@C with the hand-written adjoint (ln_gemm_chain_bwd)."""

    @staticmethod
    def forward(ctx, A, B, C, form="internalized", prec="3xbf16"):
        ctx.save_for_backward(A, B, C)
        ctx.cfg = (form, prec)
        E, _ = gemm_chain(A.contiguous(), B.contiguous(), C.contiguous(), None, 1.0, 0.0, form, prec)
        return E

    @staticmethod
    def backward(ctx, gE):
        A, B, C = ctx.saved_tensors
        dA, dB, dC = gemm_chain_bwd(A.contiguous(), B.contiguous(), C.contiguous(), gE.contiguous(), *ctx.cfg)
        return dA, dB, dC, None, None


def _cov_forward(ctx, X, fwd, fwd_stats, form, prec, keep_stats):
    Xc = X.contiguous()
    if keep_stats:  # one call: the result and the statistics the adjoint reads
        out, stats = fwd_stats(Xc, form, prec)
    else:
        out, stats = fwd(Xc, form, prec), torch.empty(0, device=X.device)
    ctx.save_for_backward(Xc, stats)
    ctx.cfg = (form, prec, keep_stats)
    return out


def _cov_backward(ctx, gR, bwd):
    Xc, stats = ctx.saved_tensors
    form, prec, keep = ctx.cfg
    return bwd(Xc, gR.contiguous(), stats if keep else None, form, prec), None, None, None


class CovarianceFn(torch.autograd.Function):
    """cov(X) with the hand-written adjoint; the centred matrix is recomputed
    from X in the backward pass instead of being stored."""

    @staticmethod
    def forward(ctx, X, form="internalized", prec="3xbf16", keep_stats=True):
        return _cov_forward(ctx, X, covariance, covariance_fwd, form, prec, keep_stats)

    @staticmethod
    def backward(ctx, gR):
        return _cov_backward(ctx, gR, covariance_bwd)


class CorrelationFn(torch.autograd.Function):
    """corr(X) with the hand-written adjoint; Z = Xc/s is recomputed from X."""

    @staticmethod
    def forward(ctx, X, form="internalized", prec="3xbf16", keep_stats=True):
        return _cov_forward(ctx, X, correlation, correlation_fwd, form, prec, keep_stats)

    @staticmethod
    def backward(ctx, gR):
        return _cov_backward(ctx, gR, correlation_bwd)
