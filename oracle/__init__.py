"""FP64 CPU oracle for the loop nests of loop internalization (paper Sec. VI-B, VI-C).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` leg may import this module;
the library under ``paper_2312_13170_gb300`` never does, and this module never
imports it. The arithmetic lives in ``oracle.c`` (plain FP64 loops); this file
only compiles it (``build()``) and marshals NumPy arrays through ctypes.

Every function takes NumPy arrays (any float dtype; widened exactly to
float64, C-contiguous) and returns float64 arrays.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

FILL_FULL, FILL_LOWER, FILL_UPPER = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc -O2 (OpenMP when available); return the .so path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = [cc, "-O2", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    d, i, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    sig = {
        "oracle_set_threads": (None, [i]),
        "oracle_max_threads": (i, []),
        "oracle_gemm": (None, [i, i, i, d, P, P, d, P, P]),
        "oracle_gemm_chain": (None, [i, i, i, i, d, P, P, P, d, P, P, P, P]),
        "oracle_3mm": (None, [i, i, i, i, i, P, P, P, P, P, P, P]),
        "oracle_3mm_vjp": (None, [i, i, i, i, i, P, P, P, P, P, P, P, P, P]),
        "oracle_col_stats": (None, [i, i, P, P, P]),
        "oracle_covariance": (None, [i, i, P, P]),
        "oracle_correlation": (None, [i, i, P, P]),
        "oracle_syrk": (None, [i, i, i, d, P, d, P, P]),
        "oracle_syr2k": (None, [i, i, i, d, P, P, d, P, P]),
        "oracle_gemm_chain_vjp": (None, [i, i, i, i, P, P, P, P, P, P, P]),
        "oracle_covariance_vjp": (None, [i, i, P, P, P]),
        "oracle_correlation_vjp": (None, [i, i, P, P, P]),
        "oracle_cov_rows": (None, [i, i, P, i, i, P, P]),
        "oracle_gramschmidt": (None, [i, i, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def gemm(A, B, C=None, alpha=1.0, beta=0.0):
    """C_out = alpha*A@B + beta*C (C not read when beta == 0)."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    Cin = _f64(C) if (C is not None and beta != 0.0) else None
    out = np.empty((M, N), np.float64)
    _load().oracle_gemm(M, N, K, float(alpha), _p(A), _p(B), float(beta), _p(Cin), _p(out))
    return out


def gemm_chain(A, B, C, D=None, alpha=1.0, beta=0.0, return_T=False):
    """T = A@B, E = T@C, F = alpha*E + beta*D. Returns (E, F) or (E, F, T)."""
    A, B, C = _f64(A), _f64(B), _f64(C)
    ni, nk = A.shape
    nj = B.shape[1]
    nl = C.shape[1]
    assert B.shape[0] == nk and C.shape[0] == nj
    Dp = _f64(D) if (D is not None and beta != 0.0) else None
    T = np.empty((ni, nj), np.float64)
    E = np.empty((ni, nl), np.float64)
    F = np.empty((ni, nl), np.float64)
    _load().oracle_gemm_chain(ni, nj, nk, nl, float(alpha), _p(A), _p(B), _p(C), float(beta),
                              _p(Dp), _p(T), _p(E), _p(F))
    return (E, F, T) if return_T else (E, F)


def three_mm(A, B, C, D, return_EF=False):
    """E = A@B, F = C@D, G = E@F (polybench 3mm). Returns G or (G, E, F)."""
    A, B, C, D = _f64(A), _f64(B), _f64(C), _f64(D)
    ni, nk = A.shape
    nj = B.shape[1]
    nm = C.shape[1]
    nl = D.shape[1]
    assert B.shape[0] == nk and C.shape[0] == nj and D.shape[0] == nm
    E = np.empty((ni, nj), np.float64)
    F = np.empty((nj, nl), np.float64)
    G = np.empty((ni, nl), np.float64)
    _load().oracle_3mm(ni, nj, nk, nl, nm, _p(A), _p(B), _p(C), _p(D), _p(E), _p(F), _p(G))
    return (G, E, F) if return_EF else G


def three_mm_vjp(A, B, C, D, Gb):
    """(dA, dB, dC, dD) for G = (A@B)@(C@D) with upstream gradient Gb = dL/dG."""
    A, B, C, D, Gb = _f64(A), _f64(B), _f64(C), _f64(D), _f64(Gb)
    ni, nk = A.shape
    nj = B.shape[1]
    nm = C.shape[1]
    nl = D.shape[1]
    out = [np.empty(s, np.float64) for s in ((ni, nk), (nk, nj), (nj, nm), (nm, nl))]
    _load().oracle_3mm_vjp(ni, nj, nk, nl, nm, _p(A), _p(B), _p(C), _p(D), _p(Gb), *(_p(x) for x in out))
    return tuple(out)


def col_stats(X):
    """Two-pass column mean and sum of squared deviations of X (n x m)."""
    X = _f64(X)
    n, m = X.shape
    mean = np.empty(m, np.float64)
    ss = np.empty(m, np.float64)
    _load().oracle_col_stats(n, m, _p(X), _p(mean), _p(ss))
    return mean, ss


def covariance(X):
    X = _f64(X)
    n, m = X.shape
    out = np.empty((m, m), np.float64)
    _load().oracle_covariance(n, m, _p(X), _p(out))
    return out


def correlation(X):
    X = _f64(X)
    n, m = X.shape
    out = np.empty((m, m), np.float64)
    _load().oracle_correlation(n, m, _p(X), _p(out))
    return out


def syrk(A, C, alpha=1.0, beta=0.0, fill=FILL_FULL):
    A, C = _f64(A), _f64(C)
    n, k = A.shape
    out = np.empty((n, n), np.float64)
    _load().oracle_syrk(int(fill), n, k, float(alpha), _p(A), float(beta), _p(C), _p(out))
    return out


def syr2k(A, B, C, alpha=1.0, beta=0.0, fill=FILL_FULL):
    A, B, C = _f64(A), _f64(B), _f64(C)
    n, k = A.shape
    assert B.shape == (n, k)
    out = np.empty((n, n), np.float64)
    _load().oracle_syr2k(int(fill), n, k, float(alpha), _p(A), _p(B), float(beta), _p(C), _p(out))
    return out


def gemm_chain_vjp(A, B, C, G):
    """(dA, dB, dC) for E = (A@B)@C with upstream gradient G = dL/dE."""
    A, B, C, G = _f64(A), _f64(B), _f64(C), _f64(G)
    ni, nk = A.shape
    nj = B.shape[1]
    nl = C.shape[1]
    dA = np.empty((ni, nk), np.float64)
    dB = np.empty((nk, nj), np.float64)
    dC = np.empty((nj, nl), np.float64)
    _load().oracle_gemm_chain_vjp(ni, nj, nk, nl, _p(A), _p(B), _p(C), _p(G), _p(dA), _p(dB), _p(dC))
    return dA, dB, dC


def covariance_vjp(X, W):
    X, W = _f64(X), _f64(W)
    n, m = X.shape
    dX = np.empty((n, m), np.float64)
    _load().oracle_covariance_vjp(n, m, _p(X), _p(W), _p(dX))
    return dX


def correlation_vjp(X, W):
    X, W = _f64(X), _f64(W)
    n, m = X.shape
    dX = np.empty((n, m), np.float64)
    _load().oracle_correlation_vjp(n, m, _p(X), _p(W), _p(dX))
    return dX


def cov_rows(X, rows, corr=False):
    """Rows `rows` of covariance (or correlation) of X, by the same definition."""
    X = _f64(X)
    n, m = X.shape
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int32))
    out = np.empty((len(r), m), np.float64)
    _load().oracle_cov_rows(n, m, _p(X), 1 if corr else 0, len(r), _p(r), _p(out))
    return out


def gramschmidt(A):
    """(Q, R) of modified Gram-Schmidt on A (m x n), polybench gramschmidt order."""
    A = _f64(A)
    m, n = A.shape
    Q = np.empty((m, n), np.float64)
    R = np.empty((n, n), np.float64)
    _load().oracle_gramschmidt(m, n, _p(A), _p(Q), _p(R))
    return Q, R
