"""Pins for the FP64 oracle, independent of the oracle itself (CPU only).

Each kernel is pinned by (a) exact rational brute force on tiny inputs,
(b) closed forms and invariants that the mathematics fixes, and (c) for the
vector-Jacobian products, exact directional derivatives (the chain is
multilinear) or FP64 central finite differences. The definitions being pinned
are the plain loop nests of paper Sec. VI-C (Listing 5) and the polybench
kernels named in Sec. VIII.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2312_13170_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore")


def F(x):
    return [[Fraction(float(v)) for v in row] for row in np.asarray(x, dtype=np.float64)]


def fmat(rows, cols, seed, lo=-1.0, hi=1.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(rows, cols)).astype(np.float32)


def exact_mm(A, B):
    n, k = len(A), len(A[0])
    m = len(B[0])
    return [[sum(A[i][q] * B[q][j] for q in range(k)) for j in range(m)] for i in range(n)]


def close(y, ref, tol=1e-14):
    y = np.asarray(y, np.float64)
    ref = np.asarray([[float(v) for v in r] for r in ref], np.float64) if isinstance(ref, list) else ref
    scale = max(1.0, float(np.max(np.abs(ref))))
    return float(np.max(np.abs(y - ref))) <= tol * scale


# ---------------------------------------------------------------- exact brute force
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (3, 5, 4), (8, 7, 6), (2, 8, 1)])
def test_gemm_exact_bruteforce(M, N, K):
    A, B, C = fmat(M, K, 1), fmat(K, N, 2), fmat(M, N, 3)
    alpha, beta = 1.5, 1.2
    ref = exact_mm(F(A), F(B))
    ref = [[Fraction(alpha) * ref[i][j] + Fraction(beta) * F(C)[i][j] for j in range(N)] for i in range(M)]
    assert close(oracle.gemm(A, B, C, alpha, beta), ref)


def test_gemm_k0_and_beta0():
    A = np.zeros((3, 0), np.float32)
    B = np.zeros((0, 4), np.float32)
    C = fmat(3, 4, 5)
    assert np.array_equal(oracle.gemm(A, B, C, 1.5, 1.2), C.astype(np.float64) * 1.2)
    C_nan = np.full((3, 4), np.nan, np.float32)
    out = oracle.gemm(fmat(3, 2, 1), fmat(2, 4, 2), C_nan, 1.0, 0.0)
    assert np.all(np.isfinite(out))  # beta == 0: C is never read


@pytest.mark.parametrize("ni,nj,nk,nl", [(2, 3, 4, 5), (6, 6, 6, 6), (1, 7, 2, 3)])
def test_chain_exact_bruteforce(ni, nj, nk, nl):
    A, B, C, D = fmat(ni, nk, 1), fmat(nk, nj, 2), fmat(nj, nl, 3), fmat(ni, nl, 4)
    alpha, beta = 1.5, 1.2
    T = exact_mm(F(A), F(B))
    E = exact_mm(T, F(C))
    Fx = [[Fraction(alpha) * E[i][l] + Fraction(beta) * F(D)[i][l] for l in range(nl)] for i in range(ni)]
    e, f, t = oracle.gemm_chain(A, B, C, D, alpha, beta, return_T=True)
    assert close(t, T) and close(e, E) and close(f, Fx)


@pytest.mark.parametrize("ni,nj,nk,nl,nm", [(1, 1, 1, 1, 1), (3, 4, 2, 5, 3), (6, 2, 5, 4, 7), (2, 7, 3, 1, 4)])
def test_3mm_exact_bruteforce(ni, nj, nk, nl, nm):
    A, B, C, D = fmat(ni, nk, 11), fmat(nk, nj, 12), fmat(nj, nm, 13), fmat(nm, nl, 14)
    E = exact_mm(F(A), F(B))
    Fm = exact_mm(F(C), F(D))
    G = exact_mm(E, Fm)
    g, e, f = oracle.three_mm(A, B, C, D, return_EF=True)
    assert close(e, E) and close(f, Fm) and close(g, G)


def exact_cov(X):
    Xf = F(X)
    n, m = len(Xf), len(Xf[0])
    mu = [sum(Xf[r][j] for r in range(n)) / n for j in range(m)]
    Xc = [[Xf[r][j] - mu[j] for j in range(m)] for r in range(n)]
    S = [[sum(Xc[r][i] * Xc[r][j] for r in range(n)) for j in range(m)] for i in range(m)]
    return mu, Xc, S


@pytest.mark.parametrize("n,m", [(2, 1), (5, 3), (8, 8), (3, 7)])
def test_covariance_exact_bruteforce(n, m):
    X = fmat(n, m, 7, -5, 5)
    _, _, S = exact_cov(X)
    ref = [[S[i][j] / (n - 1) for j in range(m)] for i in range(m)]
    assert close(oracle.covariance(X), ref)


@pytest.mark.parametrize("n,m", [(2, 2), (5, 3), (8, 8), (4, 6)])
def test_correlation_exact_bruteforce(n, m):
    X = fmat(n, m, 8, -5, 5)
    _, _, S = exact_cov(X)
    ref = np.empty((m, m))
    for i in range(m):
        for j in range(m):
            if i == j:
                ref[i, j] = 1.0
            else:
                q = S[i][j] * S[i][j] / (S[i][i] * S[j][j])  # exact rational corr^2
                ref[i, j] = math.copysign(math.sqrt(float(q)), float(S[i][j]))
    assert np.max(np.abs(oracle.correlation(X) - ref)) < 1e-14


@pytest.mark.parametrize("fill", [oracle.FILL_FULL, oracle.FILL_LOWER, oracle.FILL_UPPER])
@pytest.mark.parametrize("n,k", [(1, 1), (5, 3), (8, 8), (4, 7)])
def test_syrk_syr2k_exact_bruteforce(fill, n, k):
    A, B, C = fmat(n, k, 1), fmat(n, k, 2), fmat(n, n, 3)
    alpha, beta = 1.5, 1.2
    Af, Bf, Cf = F(A), F(B), F(C)
    a, b = Fraction(alpha), Fraction(beta)

    def expect(val):
        out = [[Cf[i][j] for j in range(n)] for i in range(n)]
        for i in range(n):
            for j in range(n):
                lower = i >= j
                if fill == oracle.FILL_UPPER:
                    if i <= j:
                        out[i][j] = a * val(i, j) + b * Cf[i][j]
                elif lower:
                    out[i][j] = a * val(i, j) + b * Cf[i][j]
        if fill == oracle.FILL_FULL:
            for i in range(n):
                for j in range(i):
                    out[j][i] = out[i][j]
        return out

    rk = expect(lambda i, j: sum(Af[i][q] * Af[j][q] for q in range(k)))
    r2k = expect(lambda i, j: sum(Af[i][q] * Bf[j][q] + Bf[i][q] * Af[j][q] for q in range(k)))
    assert close(oracle.syrk(A, C, alpha, beta, fill), rk)
    assert close(oracle.syr2k(A, B, C, alpha, beta, fill), r2k)


# ---------------------------------------------------------------- second implementation
def test_against_numpy_blas():
    A, B, C = fmat(64, 48, 1), fmat(48, 80, 2), fmat(64, 80, 3)
    Ad, Bd, Cd = (x.astype(np.float64) for x in (A, B, C))
    assert np.allclose(oracle.gemm(A, B, C, 1.5, 1.2), 1.5 * Ad @ Bd + 1.2 * Cd, rtol=0, atol=1e-12)
    X = inputs.cov_inputs(300, 40, seed=3)["X"]
    assert np.allclose(oracle.covariance(X), np.cov(X.astype(np.float64), rowvar=False), rtol=1e-12, atol=1e-12)
    R = np.corrcoef(X.astype(np.float64), rowvar=False)
    assert np.max(np.abs(oracle.correlation(X) - R)) < 1e-12


# ---------------------------------------------------------------- closed forms
def test_gemm_identity_permutation_rank1():
    n = 33
    B, C = fmat(n, n, 1), fmat(n, n, 2)
    eye = np.eye(n, dtype=np.float32)
    assert np.array_equal(oracle.gemm(eye, B, C, 1.5, 1.2), 1.5 * B.astype(np.float64) + 1.2 * C.astype(np.float64))
    perm = np.random.default_rng(0).permutation(n)
    P = eye[perm]
    assert np.array_equal(oracle.gemm(P, B), B.astype(np.float64)[perm])
    u = np.arange(1, n + 1, dtype=np.float32)
    w = np.arange(n, 0, -1, dtype=np.float32)
    K = 17
    A1 = np.repeat(u[:, None], K, axis=1)
    B1 = np.repeat(w[None, :], K, axis=0)
    assert np.array_equal(oracle.gemm(A1, B1), K * np.outer(u, w).astype(np.float64))


def test_chain_associativity_and_identity():
    A, B, C = fmat(40, 30, 1), fmat(30, 20, 2), fmat(20, 50, 3)
    E, _ = oracle.gemm_chain(A, B, C)
    BC = oracle.gemm(B, C)
    assert np.max(np.abs(E - oracle.gemm(A, BC))) < 1e-12
    E2, F2 = oracle.gemm_chain(A, B, np.eye(20, dtype=np.float32), fmat(40, 20, 4), 2.0, 0.5)
    AB = oracle.gemm(A, B)
    assert np.array_equal(E2, AB)
    assert np.array_equal(F2, 2.0 * AB + 0.5 * fmat(40, 20, 4).astype(np.float64))


def test_3mm_associativity_identity_and_rank1():
    """G = (A B)(C D) = A (B (C D)) up to rounding; C = I reduces 3mm to the
    2mm chain (A B) D exactly; rank-one factors have a closed form."""
    A, B, C, D = fmat(20, 15, 1), fmat(15, 12, 2), fmat(12, 18, 3), fmat(18, 9, 4)
    G = oracle.three_mm(A, B, C, D)
    Ad, Bd, Cd, Dd = (x.astype(np.float64) for x in (A, B, C, D))
    assert np.max(np.abs(G - Ad @ (Bd @ (Cd @ Dd)))) < 1e-12 * max(1.0, np.max(np.abs(G)))
    I = np.eye(12, dtype=np.float32)
    G2 = oracle.three_mm(A, B, I, fmat(12, 9, 5))
    E2, _ = oracle.gemm_chain(A, B, fmat(12, 9, 5))
    assert np.array_equal(G2, E2)
    # A = u 1^T, B = 1 v^T, C = 1 w^T, D = 1 y^T (all-ones inner vectors):
    # A B = nk u v^T, C D = nm 1 y^T, G = nk nm (v . 1) u y^T
    ni, nk, nj, nm, nl = 4, 3, 5, 2, 6
    u, v, y = fmat(ni, 1, 6), fmat(1, nj, 7), fmat(1, nl, 8)
    A = np.repeat(u, nk, axis=1)
    B = np.repeat(v, nk, axis=0)
    C = np.ones((nj, nm), np.float32)
    D = np.repeat(y, nm, axis=0)
    G = oracle.three_mm(A, B, C, D)
    ref = nk * nm * float(np.sum(v.astype(np.float64))) * (u.astype(np.float64) @ y.astype(np.float64))
    assert np.max(np.abs(G - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_covariance_invariants():
    X = inputs.cov_inputs(512, 24, seed=1)["X"]
    cov = oracle.covariance(X)
    assert np.array_equal(cov, cov.T)
    ev = np.linalg.eigvalsh(cov)
    assert ev.min() >= -1e-12 * np.linalg.norm(cov)
    assert np.allclose(np.diag(cov), np.var(X.astype(np.float64), axis=0, ddof=1), rtol=1e-12, atol=0)
    # shift invariance: X + 100 in every column (exact in FP64 for these FP32 values)
    Xs = X.astype(np.float64) + 100.0
    assert np.max(np.abs(oracle.covariance(Xs) - cov)) < 1e-10 * np.max(np.abs(cov))
    # closed form: each column alternates mean +/- delta over an even n
    n, d = 10, 0.25
    col = np.array([3.0 + d * (1 if r % 2 == 0 else -1) for r in range(n)])
    Xa = np.stack([col, 2 * col], axis=1)
    cv = oracle.covariance(Xa)
    assert abs(cv[0, 0] - d * d * n / (n - 1)) < 1e-15
    assert abs(cv[1, 1] - 4 * d * d * n / (n - 1)) < 1e-15
    assert abs(cv[0, 1] - 2 * d * d * n / (n - 1)) < 1e-15


def test_correlation_invariants():
    X = inputs.cov_inputs(256, 12, seed=2)["X"].astype(np.float64)
    R = oracle.correlation(X)
    assert np.all(np.diag(R) == 1.0)
    assert np.max(np.abs(R)) <= 1.0 + 1e-15
    assert np.array_equal(R, R.T)
    scale = np.exp(np.linspace(-3, 3, 12))
    R2 = oracle.correlation(X * scale[None, :] - 7.0)
    assert np.max(np.abs(R2 - R)) < 1e-10
    Xd = np.concatenate([X[:, :3], X[:, :1], -X[:, 1:2]], axis=1)
    Rd = oracle.correlation(Xd)
    assert abs(Rd[0, 3] - 1.0) < 1e-14 and abs(Rd[1, 4] + 1.0) < 1e-14
    # zero-variance column: off-diagonal zero, diagonal one
    Xz = X[:, :4].copy()
    Xz[:, 2] = 5.0
    Rz = oracle.correlation(Xz)
    assert np.all(Rz[2, [0, 1, 3]] == 0.0) and np.all(Rz[[0, 1, 3], 2] == 0.0) and Rz[2, 2] == 1.0


def test_syrk_syr2k_identities():
    A, B = fmat(30, 20, 1), fmat(30, 20, 2)
    C = inputs.sym_inputs(30, 20, seed=3)["C"]
    s = oracle.syrk(A, C, 1.5, 1.2)
    assert np.max(np.abs(s - oracle.gemm(A, A.T, C, 1.5, 1.2))) < 1e-13
    s2 = oracle.syr2k(A, B, C, 1.5, 1.2)
    ref = 1.5 * (A.astype(np.float64) @ B.T.astype(np.float64) + B.astype(np.float64) @ A.T.astype(np.float64)) + 1.2 * C.astype(np.float64)
    assert np.max(np.abs(s2 - ref)) < 1e-13
    assert np.max(np.abs(oracle.syr2k(A, A, C, 1.5, 1.2) - oracle.syrk(A, C, 3.0, 1.2))) < 1e-13
    # LOWER leaves the strict upper triangle of C untouched
    low = oracle.syrk(A, C, 1.5, 1.2, oracle.FILL_LOWER)
    iu = np.triu_indices(30, 1)
    assert np.array_equal(low[iu], C.astype(np.float64)[iu])


# ---------------------------------------------------------------- gradients
def test_chain_vjp_exact_directional():
    """E = (A B) C is linear in each factor, so <dL/dA, H> = L(A+H) - L(A) exactly."""
    ni, nj, nk, nl = 3, 4, 2, 5
    A, B, C, G = fmat(ni, nk, 1), fmat(nk, nj, 2), fmat(nj, nl, 3), fmat(ni, nl, 4)
    H = [fmat(ni, nk, 5), fmat(nk, nj, 6), fmat(nj, nl, 7)]
    dA, dB, dC = oracle.gemm_chain_vjp(A, B, C, G)

    def L(a, b, c):
        E = exact_mm(exact_mm(F(a), F(b)), F(c))
        Gf = F(G)
        return sum(Gf[i][l] * E[i][l] for i in range(ni) for l in range(nl))

    base = L(A, B, C)
    for grad, idx in ((dA, 0), (dB, 1), (dC, 2)):
        args = [A.astype(np.float64), B.astype(np.float64), C.astype(np.float64)]
        args[idx] = args[idx] + H[idx].astype(np.float64)
        exact = float(L(*args) - base)
        got = float(np.sum(grad * H[idx].astype(np.float64)))
        assert abs(got - exact) <= 1e-13 * max(1.0, abs(exact))


def test_3mm_vjp_exact_directional():
    """G = (A B)(C D) is linear in each factor, so <dL/dX, H> = L(X+H) - L(X)
    exactly for L = <Gb, G> and any one factor X. The adjoint of a plausible
    mistake, G' = (A B)(C D)^T (F transposed, square factors), must fail it."""
    ni, nj, nk, nl, nm = 3, 4, 2, 4, 4
    A, B, C, D, Gb = fmat(ni, nk, 1), fmat(nk, nj, 2), fmat(nj, nm, 3), fmat(nm, nl, 4), fmat(ni, nl, 5)
    H = [fmat(ni, nk, 6), fmat(nk, nj, 7), fmat(nj, nm, 8), fmat(nm, nl, 9)]

    def L(a, b, c, d):
        G = exact_mm(exact_mm(F(a), F(b)), exact_mm(F(c), F(d)))
        Gf = F(Gb)
        return sum(Gf[i][l] * G[i][l] for i in range(ni) for l in range(nl))

    base_args = [x.astype(np.float64) for x in (A, B, C, D)]
    base = L(*base_args)

    def matches(grads):
        for idx, grad in enumerate(grads):
            args = list(base_args)
            args[idx] = args[idx] + H[idx].astype(np.float64)
            exact = float(L(*args) - base)
            got = float(np.sum(grad * H[idx].astype(np.float64)))
            if abs(got - exact) > 1e-13 * max(1.0, abs(exact)):
                return False
        return True

    assert matches(oracle.three_mm_vjp(A, B, C, D, Gb))
    # (C D)^T = D^T C^T: the adjoint of E (D^T C^T) in place of E (C D)
    wrong = oracle.three_mm_vjp(A, B, np.ascontiguousarray(D.T), np.ascontiguousarray(C.T), Gb)
    assert not matches((wrong[0], wrong[1], np.ascontiguousarray(wrong[3].T), np.ascontiguousarray(wrong[2].T)))


def _fd_check(fun, X, dX, h_rel=1e-6, tol=1e-7, seed=0):
    rng = np.random.default_rng(seed)
    n, m = X.shape
    errs = []
    for _ in range(12):
        r, c = int(rng.integers(n)), int(rng.integers(m))
        h = h_rel * max(1.0, abs(X[r, c]))
        Xp, Xm = X.copy(), X.copy()
        Xp[r, c] += h
        Xm[r, c] -= h
        fd = (fun(Xp) - fun(Xm)) / (2 * h)
        errs.append(abs(fd - dX[r, c]) / max(1e-3, np.max(np.abs(dX))))
    assert max(errs) < tol, max(errs)


def test_covariance_vjp_finite_difference():
    X = inputs.backward_inputs(16, 16, 4, seed=1)["X"].astype(np.float64)
    W = fmat(16, 16, 9).astype(np.float64)
    dX = oracle.covariance_vjp(X, W)
    _fd_check(lambda Y: float(np.sum(W * oracle.covariance(Y))), X, dX)
    assert np.max(np.abs(dX.sum(axis=0))) < 1e-12 * np.max(np.abs(dX)) * 16


def test_correlation_vjp_finite_difference():
    X = inputs.backward_inputs(16, 16, 4, seed=2)["X"].astype(np.float64)
    W = fmat(16, 16, 10).astype(np.float64)
    dX = oracle.correlation_vjp(X, W)
    _fd_check(lambda Y: float(np.sum(W * oracle.correlation(Y))), X, dX)
    assert np.max(np.abs(dX.sum(axis=0))) < 1e-12 * np.max(np.abs(dX)) * 16
    # diagonal-only upstream gradient: corr_ii = 1 is constant, so dX = 0
    assert np.max(np.abs(oracle.correlation_vjp(X, np.diag(np.arange(16.0))))) < 1e-14


def test_chain_vjp_finite_difference_frobenius_loss():
    """L = ||(AB)C||_F^2 has dL/dE = 2E; check dA by central differences at n = 16."""
    d = inputs.backward_inputs(16, 4, 16, seed=3)
    A, B, C = (d[k].astype(np.float64) for k in "ABC")
    E, _ = oracle.gemm_chain(A, B, C)
    dA, dB, dC = oracle.gemm_chain_vjp(A, B, C, 2.0 * E)

    def L(a, b, c):
        return float(np.sum(oracle.gemm_chain(a, b, c)[0] ** 2))

    _fd_check(lambda Y: L(Y, B, C), A, dA)
    _fd_check(lambda Y: L(A, Y, C), B, dB)
    _fd_check(lambda Y: L(A, B, Y), C, dC)


# ---------------------------------------------------------------- the pins catch planted mistakes
def test_pins_reject_planted_mistakes():
    """A transposed operand, a dropped beta term or a wrong divisor must fail the
    exact brute-force pins above (the mistake is planted here, on the CPU)."""
    n = 6
    A, B, C = fmat(n, n, 1), fmat(n, n, 2), fmat(n, n, 3)
    ref = exact_mm(F(A), F(B))
    ref = [[Fraction(1.5) * ref[i][j] + Fraction(1.2) * F(C)[i][j] for j in range(n)] for i in range(n)]
    assert not close(oracle.gemm(A, B.T.copy(), C, 1.5, 1.2), ref)
    assert not close(oracle.gemm(A, B, C, 1.5, 0.0), ref)
    X = fmat(8, 4, 7, -5, 5)
    _, _, S = exact_cov(X)
    wrong = [[S[i][j] / 8 for j in range(4)] for i in range(4)]  # divisor n instead of n-1
    assert not close(oracle.covariance(X), wrong)
    # 3mm with a transposed F (E F^T) or with the factors swapped (F E) must miss
    A, B, Cm, Dm = fmat(n, n, 4), fmat(n, n, 5), fmat(n, n, 6), fmat(n, n, 8)
    G = exact_mm(exact_mm(F(A), F(B)), exact_mm(F(Cm), F(Dm)))
    assert not close(oracle.three_mm(A, B, Dm.T.copy(), Cm.T.copy()), G)
    assert not close(oracle.three_mm(Cm, Dm, A, B), G)


def test_cov_rows_matches_full():
    X = inputs.cov_inputs(64, 20, seed=4)["X"]
    rows = [0, 7, 19, 3]
    assert np.array_equal(oracle.cov_rows(X, rows), oracle.covariance(X)[rows])
    assert np.array_equal(oracle.cov_rows(X, rows, corr=True), oracle.correlation(X)[rows])


@pytest.mark.parametrize("n,m", [(1, 1), (2, 3), (5, 4), (8, 2)])
def test_col_stats_exact_fraction(n, m):
    """oracle.col_stats (mean, ss) against exact rational arithmetic: entries are
    multiples of 1/8, so every sum is exact in FP64 and the mean is the exact
    quotient rounded once; ss = sum (x - mean)^2 is within a few ulps of the
    exact value. A swapped (ss, mean) return, a dropped centring or a divisor
    in ss fails."""
    rng = np.random.default_rng(n * 10 + m)
    X = (rng.integers(-80, 80, size=(n, m)) / 8.0).astype(np.float32)
    X[:, 0] += 100.0  # one column far from zero: centring matters
    mean, ss = oracle.col_stats(X)
    for j in range(m):
        col = [Fraction(float(v)) for v in X[:, j]]
        mu = sum(col) / n
        s2 = sum((x - mu) ** 2 for x in col)
        assert mean[j] == float(mu)
        assert abs(Fraction(float(ss[j])) - s2) <= Fraction(1, 10 ** 12) * max(s2, Fraction(1, 64)), (j, ss[j], s2)
    # the same statistics as the definition computed by NumPy in FP64
    X64 = X.astype(np.float64)
    assert np.allclose(ss, ((X64 - X64.mean(axis=0)) ** 2).sum(axis=0), rtol=1e-12, atol=1e-12)
