"""GPU parity of Gram-Schmidt QR (polybench gramschmidt) against the FP64 oracle.

Both forms compute in FP32. Bounds, from the arithmetic: R and the residual
A - QR are backward-stable quantities, gated at 1e-5 relative Frobenius like
the rest of the library; the forward error of Q of any Gram-Schmidt variant
grows with the condition number (loss of orthogonality ~ kappa * u), so Q is
gated at max(1e-5, kappa_2(A) * 2^-24) with kappa from an FP64 SVD of the
input. Sizes cover one and several 32-column panels with ragged last panels,
every panel kernel (registers with 2 or 4 rows per thread, shared memory,
L2), zero columns, empty shapes, in-place use and graph replay.
"""
import numpy as np
import pytest

import oracle
from paper_2312_13170_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = 1e-5
FORMS = ["plain", "internalized"]


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2312_13170_gb300 import api as a

    return a


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def check(A, Q, R, Qo, Ro):
    kappa = np.linalg.cond(A.astype(np.float64))
    assert np.array_equal(np.tril(R, -1), np.zeros_like(R)), "R must be upper triangular"
    assert np.all(np.diag(R) >= 0)
    assert inputs.rel_fro(R, Ro) <= GATE
    assert inputs.rel_fro(Q, Qo) <= max(GATE, kappa * 2.0 ** -24)
    assert inputs.rel_fro(Q @ R, A.astype(np.float64)) <= GATE


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (33, 33), (65, 40), (200, 136), (300, 300), (513, 200),
                                 (1024, 1024), (1500, 100), (2100, 70)])
def test_gramschmidt(api, form, m, n):
    if form == "plain" and m * n > 300 * 300 and m < 1024:
        pytest.skip("the plain form is covered at the other sizes")
    A = inputs.gramschmidt_inputs(m, n, seed=m + n)["A"]
    Qo, Ro = oracle.gramschmidt(A)
    Q, R = api.gramschmidt(dev(A), form=form)
    api.stream_check()
    check(A, host(Q), host(R), Qo, Ro)


@pytest.mark.parametrize("rows", [2, 4])
def test_gramschmidt_panel_rows_knob(api, rows):
    A = inputs.gramschmidt_inputs(700, 96, seed=3)["A"]
    Qo, Ro = oracle.gramschmidt(A)
    old = api.get_tuning("gs_rows")
    try:
        api.set_tuning("gs_rows", rows)
        Q, R = api.gramschmidt(dev(A))
        api.stream_check()
    finally:
        api.set_tuning("gs_rows", old)
    check(A, host(Q), host(R), Qo, Ro)


@pytest.mark.parametrize("form", FORMS)
def test_gramschmidt_zero_column_and_triangular(api, form):
    A = inputs.gramschmidt_inputs(90, 40, seed=5)["A"]
    A[:, 3] = 0.0
    A[:, 35] = 0.0
    Q, R = api.gramschmidt(dev(A), form=form)
    api.stream_check()
    Q, R = host(Q), host(R)
    for c in (3, 35):
        assert np.array_equal(Q[:, c], np.zeros(90)) and np.array_equal(R[c], np.zeros(40))
    keep = [j for j in range(40) if j not in (3, 35)]
    Qo, Ro = oracle.gramschmidt(A[:, keep])
    check(A[:, keep], Q[:, keep], R[np.ix_(keep, keep)], Qo, Ro)
    # an upper-triangular matrix with a positive diagonal is its own R, with Q = I
    T = np.triu(inputs.gramschmidt_inputs(48, 48, seed=6)["A"])
    T[np.diag_indices(48)] = np.abs(T[np.diag_indices(48)]) + 0.5
    Q, R = api.gramschmidt(dev(T), form=form)
    api.stream_check()
    if form == "plain":  # q = a/a = 1 and R[k][j] = 1 * a exactly: Q = I and R = T bit for bit
        assert np.array_equal(host(Q), np.eye(48)) and np.array_equal(host(R), T)
    else:  # inside a panel R[k][j] = (a_kk a_kj) / a_kk, which may miss a_kj by an ulp, and random
        # triangular matrices are badly conditioned, so only the conditioning-scaled bounds hold
        check(T, host(Q), host(R), np.eye(48), T.astype(np.float64))


@pytest.mark.parametrize("form", FORMS)
def test_gramschmidt_empty_in_place_and_deterministic(api, form):
    R = dev(np.full((6, 6), np.nan, np.float32))
    Q, R = api.gramschmidt(dev(np.zeros((0, 6), np.float32)), form=form, R=R)
    assert np.array_equal(host(R), np.zeros((6, 6)))
    Q, R = api.gramschmidt(dev(np.zeros((7, 0), np.float32)), form=form)
    assert tuple(Q.shape) == (7, 0) and tuple(R.shape) == (0, 0)
    A = inputs.gramschmidt_inputs(260, 90, seed=7)["A"]
    Q1, R1 = api.gramschmidt(dev(A), form=form)
    Q2, R2 = api.gramschmidt(dev(A), form=form)
    Ad = dev(A)
    Q3, R3 = api.gramschmidt(Ad, form=form, in_place=True)
    api.stream_check()
    assert Q3.data_ptr() == Ad.data_ptr()
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2) and torch.equal(Q1, Q3) and torch.equal(R1, R3)


def test_gramschmidt_graph_replay(api):
    A = inputs.gramschmidt_inputs(1024, 1024, seed=0)["A"]
    Ad = dev(A)
    Q = torch.empty_like(Ad)
    R = torch.empty((1024, 1024), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        api.gramschmidt(Ad, Q=Q, R=R, stream=s)  # warm-up outside the capture
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            api.gramschmidt(Ad, Q=Q, R=R, stream=s)
    Qe, Re = host(Q).copy(), host(R).copy()
    Q.fill_(np.nan)
    R.fill_(np.nan)
    g.replay()
    api.stream_check()
    assert np.array_equal(host(Q), Qe) and np.array_equal(host(R), Re)
    Qo, Ro = oracle.gramschmidt(A)
    check(A, Qe, Re, Qo, Ro)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("m,n", [(300, 100), (1100, 70)])
def test_gramschmidt_strided_unaligned(api, form, m, n):
    # leading dimensions that are not multiples of 4: the scalar fill, write-out and staging paths
    A = inputs.gramschmidt_inputs(m, n, seed=11)["A"]
    Qo, Ro = oracle.gramschmidt(A)
    big = torch.full((m, n + 3), float("nan"), dtype=torch.float32, device="cuda")
    big[:, 1:n + 1] = dev(A)
    Av = big[:, 1:n + 1]
    Qbig = torch.full((m, n + 5), float("nan"), dtype=torch.float32, device="cuda")
    Rbig = torch.full((n, n + 2), float("nan"), dtype=torch.float32, device="cuda")
    Q, R = api.gramschmidt(Av, form=form, Q=Qbig[:, 2:n + 2], R=Rbig[:, 1:n + 1])
    api.stream_check()
    check(A, host(Q), host(R), Qo, Ro)
    # nothing outside the views was written
    assert torch.isnan(Qbig[:, :2]).all() and torch.isnan(Qbig[:, n + 2:]).all()
    assert torch.isnan(Rbig[:, :1]).all() and torch.isnan(Rbig[:, n + 1:]).all()
    assert torch.isnan(big[:, 0]).all() and torch.isnan(big[:, n + 1:]).all()


@pytest.mark.parametrize("form", FORMS)
def test_gramschmidt_golden(api, form):
    # the hand-derived worked example of tests/golden/hand_examples.json
    import json
    import os
    from fractions import Fraction

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")))["gramschmidt"]
    Q, R = api.gramschmidt(dev(np.array(g["A"], np.float32)), form=form)
    api.stream_check()
    Qe = np.array([[float(Fraction(x)) for x in row] for row in g["Q"]])
    Re = np.array([[float(Fraction(x)) for x in row] for row in g["R"]])
    assert np.max(np.abs(host(Q) - Qe)) <= 2 ** -22 and np.max(np.abs(host(R) - Re)) <= 13 * 2 ** -22
