"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: it only draws random numbers
(NumPy ``default_rng``, PCG64) in a fixed, documented order and returns FP32
arrays (plus the scalar parameters of each workload). Both the FP64 oracle and
the CUDA library consume exactly these arrays.

Workloads (all seeds default to 0; draws are made in the order listed,
row-major, as FP64, then cast to FP32):

* ``gemm``   C = alpha*A*B + beta*C, A/B/C ~ U[-1,1] (order A, B, C),
             alpha = 1.5, beta = 1.2.  The 256^3 case is the small oracle case.
* ``chain``  E = (A*B)*C, F = alpha*E + beta*D, A/B/C/D ~ U[-1,1]
             (order A, B, C, D), alpha = 1.5, beta = 1.2; 2048^2 in the benchmark.
* ``cov``    data matrix of n samples x m features: mean_j ~ U[-100,100],
             std_j = exp(U[ln 0.01, ln 10]), X = mean_j + std_j * N(0,1)
             (order: means, stds, then the n x m normals); 8192 x 2048.
* ``sym_batch`` batched SYRK/SYR2K: per instance n then k, each
             round(exp(U[ln lo, ln hi])) (all sizes first), then per instance
             A, B ~ U[-1,1] (n x k) and R ~ U[-1,1] (n x n), C0 = (R + R^T)/2;
             alpha = 1.5, beta = 1.2; 512 instances with n, k in [32, 1536].
* ``backward`` X (n x m) = N(0,1) * scale_j, scale_j = exp(U[ln 0.1, ln 10])
             (order: scales, X), then W (m x m), A, B, C (p x p) ~ U[-1,1];
             4096 x 1024 and p = 1024.
* ``gramschmidt`` A (m x n) ~ U[-1,1]; 1024 x 1024 in the benchmark (the
             paper's polybench size). Square uniform matrices of this size have
             a 2-norm condition number of a few thousand, so FP32 Gram-Schmidt
             loses about that factor of orthogonality (tests scale their bound
             for Q with it).

These stand in for the polybench workloads of SYCL-Bench used in the paper's
evaluation (Sec. VIII), whose sources and data are not part of this project:
only the kernels' definitions and problem shapes are taken from the paper.
"""
from __future__ import annotations

import math

import numpy as np

ALPHA = 1.5
BETA = 1.2


def _u(rng, shape, lo=-1.0, hi=1.0):
    return rng.uniform(lo, hi, size=shape).astype(np.float32)


def gemm_inputs(M=256, N=256, K=256, seed=0):
    rng = np.random.default_rng(seed)
    A = _u(rng, (M, K))
    B = _u(rng, (K, N))
    C = _u(rng, (M, N))
    return {"A": A, "B": B, "C": C, "alpha": ALPHA, "beta": BETA}


def chain_inputs(ni=2048, nj=None, nk=None, nl=None, seed=0):
    nj = ni if nj is None else nj
    nk = ni if nk is None else nk
    nl = ni if nl is None else nl
    rng = np.random.default_rng(seed)
    A = _u(rng, (ni, nk))
    B = _u(rng, (nk, nj))
    C = _u(rng, (nj, nl))
    D = _u(rng, (ni, nl))
    return {"A": A, "B": B, "C": C, "D": D, "alpha": ALPHA, "beta": BETA}


def cov_inputs(nsamples=8192, nfeat=2048, seed=0):
    rng = np.random.default_rng(seed)
    mean = rng.uniform(-100.0, 100.0, size=nfeat)
    std = np.exp(rng.uniform(math.log(0.01), math.log(10.0), size=nfeat))
    Z = rng.standard_normal(size=(nsamples, nfeat))
    X = (mean[None, :] + std[None, :] * Z).astype(np.float32)
    return {"X": X}


def sym_batch_sizes(count=512, lo=32, hi=1536, seed=0):
    """Per-instance (n, k), drawn n then k for each instance, log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), size=(count, 2))
    return np.rint(np.exp(u)).astype(np.int64), rng


def sym_batch_inputs(count=512, lo=32, hi=1536, seed=0, with_b=True):
    sizes, rng = sym_batch_sizes(count, lo, hi, seed)
    inst = []
    for n, k in sizes:
        n, k = int(n), int(k)
        A = _u(rng, (n, k))
        B = _u(rng, (n, k))
        R = rng.uniform(-1.0, 1.0, size=(n, n))
        C = ((R + R.T) * 0.5).astype(np.float32)
        inst.append({"n": n, "k": k, "A": A, "B": B if with_b else None, "C": C})
    return {"instances": inst, "alpha": ALPHA, "beta": BETA}


def sym_inputs(n=256, k=256, seed=0):
    """One SYRK/SYR2K instance: A, B ~ U[-1,1] (n x k), C = (R + R^T)/2."""
    rng = np.random.default_rng(seed)
    A = _u(rng, (n, k))
    B = _u(rng, (n, k))
    R = rng.uniform(-1.0, 1.0, size=(n, n))
    C = ((R + R.T) * 0.5).astype(np.float32)
    return {"A": A, "B": B, "C": C, "alpha": ALPHA, "beta": BETA}


def backward_inputs(nsamples=4096, nfeat=1024, p=1024, seed=0):
    rng = np.random.default_rng(seed)
    scale = np.exp(rng.uniform(math.log(0.1), math.log(10.0), size=nfeat))
    X = (rng.standard_normal(size=(nsamples, nfeat)) * scale[None, :]).astype(np.float32)
    W = _u(rng, (nfeat, nfeat))
    A = _u(rng, (p, p))
    B = _u(rng, (p, p))
    C = _u(rng, (p, p))
    return {"X": X, "W": W, "A": A, "B": B, "C": C}


def int_matrix(shape, lo=-4, hi=4, seed=0):
    """Integer-valued FP32 matrix with entries in [lo, hi]: every product and
    partial sum of the tests that use it is exact in BF16/TF32/FP32."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=shape).astype(np.float32)


def rel_fro(y, ref) -> float:
    """Relative Frobenius error ||y - ref||_F / ||ref||_F, evaluated in FP64."""
    y = np.asarray(y, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.linalg.norm(ref))
    num = float(np.linalg.norm(y - ref))
    return num / den if den > 0 else num


def gramschmidt_inputs(m=1024, n=1024, seed=0):
    rng = np.random.default_rng(seed)
    return {"A": _u(rng, (m, n))}
