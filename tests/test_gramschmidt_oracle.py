"""Pins for the FP64 Gram-Schmidt oracle (polybench gramschmidt, paper Sec. VIII),
independent of the oracle itself (CPU only).

The oracle runs modified Gram-Schmidt column by column. What pins it:
(a) exact QR of small integer matrices from SymPy's rational/radical
    arithmetic; (b) LAPACK's Householder QR (NumPy) with the signs fixed so
    that diag(R) > 0, which makes the thin QR of a full-rank matrix unique;
(c) special cases with closed forms: an upper-triangular matrix gives Q = I
    and R = A bit for bit, orthonormal columns give R = I, a scaled column
    scales its R column, a zero column gives a zero Q column and R row and
    leaves everything else as for the matrix without it; (d) the Laeuchli
    matrix, whose floating-point MGS result is known in closed form and
    differs from classical Gram-Schmidt's (the textbook example of MGS's
    better orthogonality), which pins the *modified* update order.
A planted-mistake test shows that each of these catches a plausible slip.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")


def uni(m, n, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(m, n)).astype(np.float32)


def lapack_qr(A):
    Q, R = np.linalg.qr(np.asarray(A, np.float64), mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :], R * d[:, None]


def laeuchli(eps):
    A = np.zeros((4, 3))
    A[0, :] = 1.0
    for j in range(3):
        A[j + 1, j] = eps
    return A


def laeuchli_mgs(eps):
    """MGS on the Laeuchli matrix in floating point, where 1 + eps^2 rounds to 1."""
    s2, s6 = math.sqrt(2.0), math.sqrt(6.0)
    Q = np.array([[1.0, 0.0, 0.0], [eps, -1 / s2, -1 / s6], [0.0, 1 / s2, -1 / s6], [0.0, 0.0, 2 / s6]])
    R = np.array([[1.0, 1.0, 1.0], [0.0, eps * s2, eps / s2], [0.0, 0.0, eps * math.sqrt(1.5)]])
    return Q, R


# ---- the pins, as predicates so that the planted-mistake test can reuse them
def pin_sympy(gs):
    sympy = pytest.importorskip("sympy")
    for A in ([[3, 1, 2], [4, -2, 0], [0, 5, 1], [1, 1, 7]], [[2, -1], [1, 3]], [[4, 0, 1], [1, 3, 0], [0, 1, 5]]):
        Qs, Rs = sympy.Matrix(A).QRdecomposition()
        Qe = np.array(Qs.evalf(30).tolist(), np.float64)
        Re = np.array(Rs.evalf(30).tolist(), np.float64)
        Q, R = gs(np.array(A, np.float64))
        if not (np.allclose(Q, Qe, rtol=0, atol=1e-14) and np.allclose(R, Re, rtol=0, atol=1e-13)):
            return False
    return True


def pin_lapack(gs):
    for m, n, seed in [(7, 5, 1), (40, 40, 2), (300, 200, 3)]:
        A = uni(m, n, seed)
        Q, R = gs(A)
        Ql, Rl = lapack_qr(A)
        if not (np.allclose(Q, Ql, rtol=0, atol=1e-10) and np.allclose(R, Rl, rtol=0, atol=1e-10)):
            return False
    return True


def pin_laeuchli(gs):
    eps = 1e-10
    Q, R = gs(laeuchli(eps))
    Qe, Re = laeuchli_mgs(eps)
    okR = np.all(np.abs(R - Re) <= 1e-12 * np.abs(Re) + 1e-300)
    return bool(np.allclose(Q, Qe, rtol=0, atol=1e-12) and okR and abs(Q[:, 1] @ Q[:, 2]) < 1e-12)


def pin_triangular(gs):
    rng = np.random.default_rng(4)
    A = np.triu(rng.uniform(-1, 1, (9, 9)))
    A[np.diag_indices(9)] = rng.uniform(0.5, 2.0, 9)
    Q, R = gs(A)
    return bool(np.array_equal(Q, np.eye(9)) and np.array_equal(R, A))


def pin_orthonormal_and_scaling(gs):
    U, _ = lapack_qr(uni(30, 12, 5))
    Q, R = gs(U)
    if not (np.allclose(R, np.eye(12), atol=1e-14) and np.allclose(Q, U, atol=1e-14)):
        return False
    A = uni(30, 12, 6).astype(np.float64)
    Q0, R0 = gs(A)
    As = A.copy()
    As[:, 4] *= 8.0  # a power of two: every operation on that column scales exactly
    Q1, R1 = gs(As)
    R0s = R0.copy()
    R0s[:, 4] *= 8.0
    return bool(np.allclose(Q1, Q0, atol=1e-14) and np.allclose(R1, R0s, atol=1e-13))


def pin_zero_column(gs):
    A = uni(20, 8, 7).astype(np.float64)
    A[:, 3] = 0.0
    Q, R = gs(A)
    keep = [0, 1, 2, 4, 5, 6, 7]
    Qk, Rk = gs(A[:, keep])
    return bool(
        np.array_equal(Q[:, 3], np.zeros(20)) and np.array_equal(R[3], np.zeros(8)) and np.array_equal(R[:, 3][4:], np.zeros(4))
        and np.array_equal(Q[:, keep], Qk) and np.array_equal(R[np.ix_(keep, keep)], Rk))


PINS = [pin_sympy, pin_lapack, pin_laeuchli, pin_triangular, pin_orthonormal_and_scaling, pin_zero_column]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_oracle_gramschmidt_pins(pin):
    assert pin(oracle.gramschmidt)


def test_oracle_gramschmidt_invariants_and_empty():
    A = uni(64, 48, 8)
    Q, R = oracle.gramschmidt(A)
    assert np.array_equal(np.tril(R, -1), np.zeros_like(R))
    assert np.all(np.diag(R) > 0)
    assert np.linalg.norm(Q @ R - A) <= 1e-14 * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(48)) <= 1e-13
    Q, R = oracle.gramschmidt(np.zeros((0, 5), np.float32))
    assert Q.shape == (0, 5) and np.array_equal(R, np.zeros((5, 5)))
    Q, R = oracle.gramschmidt(np.zeros((6, 0), np.float32))
    assert Q.shape == (6, 0) and R.shape == (0, 0)


# ---- planted mistakes (on the CPU, in a small pure-NumPy stand-in)
def planted(A, mistake):
    W = np.array(A, np.float64)
    m, n = W.shape
    A0 = W.copy()
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    for k in range(n):
        R[k, k] = math.sqrt(float(W[:, k] @ W[:, k]))
        Q[:, k] = W[:, k] / R[k, k] if R[k, k] > 0 else 0.0
        for j in range(k + 1, n):
            src = A0[:, j] if mistake == "classical" else W[:, j]
            R[k, j] = Q[:, k] @ src
            if mistake != "no_update":
                W[:, j] -= Q[:, k] * R[k, j]
    if mistake == "transposed_R":
        R = R.T.copy()
    if mistake == "unnormalised":
        Q = Q * np.diag(R)[None, :]
    return Q, R


@pytest.mark.parametrize("mistake", ["classical", "no_update", "transposed_R", "unnormalised"])
def test_pins_reject_planted_gramschmidt_mistakes(mistake):
    assert pin_lapack(lambda A: planted(A, None)) and pin_laeuchli(lambda A: planted(A, None))
    caught = [p.__name__ for p in PINS if not p(lambda A: planted(A, mistake))]
    assert caught, f"no pin catches the '{mistake}' mistake"
