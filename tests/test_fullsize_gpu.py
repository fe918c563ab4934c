"""Parity at the full workload sizes, in the launch configuration the
benchmark times, on outputs the oracle computes one row at a time.

Workloads: the 2048^2 chained product; covariance and correlation of an
8192 x 2048 data matrix; 512 uneven SYRK/SYR2K instances; the backward pass
of sum(W .* corr(X)) + ||(A B) C||_F^2 with X 4096 x 1024 and 1024^2 factors.
"""
import numpy as np
import pytest

import oracle
from paper_2312_13170_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GATE = 1e-5


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
    return t.detach().cpu().numpy()


ROWS = np.random.default_rng(123).choice(2048, size=12, replace=False)


@pytest.mark.parametrize("form,prec", [("internalized", "3xbf16"), ("internalized", "3xtf32"), ("internalized", "fp32"),
                                       ("plain", "fp32")])
def test_chain_2048(api, form, prec):
    d = inputs.chain_inputs(2048, seed=0)
    E, F = api.gemm_chain(dev(d["A"]), dev(d["B"]), dev(d["C"]), dev(d["D"]), d["alpha"], d["beta"],
                          form=form, prec=prec)
    api.stream_check()
    # rows of E and F depend only on the same rows of A and D
    E_ref, F_ref = oracle.gemm_chain(d["A"][ROWS], d["B"], d["C"], d["D"][ROWS], d["alpha"], d["beta"])
    assert inputs.rel_fro(host(E)[ROWS], E_ref) <= GATE
    assert inputs.rel_fro(host(F)[ROWS], F_ref) <= GATE


@pytest.mark.parametrize("form,prec", [("internalized", "3xbf16"), ("internalized", "3xtf32"), ("internalized", "fp32")])
def test_cov_corr_8192x2048(api, form, prec):
    X = inputs.cov_inputs(8192, 2048, seed=0)["X"]
    Xd = dev(X)
    cov = host(api.covariance(Xd, form=form, prec=prec))
    corr = host(api.correlation(Xd, form=form, prec=prec))
    api.stream_check()
    assert inputs.rel_fro(cov[ROWS], oracle.cov_rows(X, ROWS)) <= GATE
    assert inputs.rel_fro(corr[ROWS], oracle.cov_rows(X, ROWS, corr=True)) <= GATE
    assert np.all(np.diag(corr) == 1.0) and np.array_equal(cov, cov.T)


@pytest.mark.parametrize("two", [False, True])
def test_batched_512(api, two):
    b = inputs.sym_batch_inputs(512, 32, 1536, seed=0)
    inst = b["instances"]
    As = [dev(x["A"]) for x in inst]
    Bs = [dev(x["B"]) for x in inst] if two else None
    Cs = [dev(x["C"]) for x in inst]
    api.SymBatch(As, Cs, Bs, b["alpha"], b["beta"], prec="3xbf16").run()
    api.stream_check()
    rng = np.random.default_rng(1)
    worst = 0.0
    for x, C in zip(inst, Cs):
        rows = rng.choice(x["n"], size=min(3, x["n"]), replace=False)
        # C is symmetric, so FULL-fill rows equal rows of alpha*A A^T + beta*C (SYRK = GEMM(A, A^T))
        if two:
            ref = oracle.gemm(x["A"][rows], x["B"].T, x["C"][rows], b["alpha"], b["beta"])
            ref += oracle.gemm(x["B"][rows], x["A"].T, None, b["alpha"], 0.0)
        else:
            ref = oracle.gemm(x["A"][rows], x["A"].T, x["C"][rows], b["alpha"], b["beta"])
        worst = max(worst, inputs.rel_fro(host(C)[rows], ref))
    assert worst <= GATE, worst


def test_backward_4096x1024(api):
    d = inputs.backward_inputs(4096, 1024, 1024, seed=0)
    X = dev(d["X"]).requires_grad_(True)
    A, B, C = (dev(d[k]).requires_grad_(True) for k in "ABC")
    W = dev(d["W"])
    R = api.CorrelationFn.apply(X, "internalized", "3xbf16", True)
    E = api.GemmChainFn.apply(A, B, C, "internalized", "3xbf16")
    ((W * R).sum() + (E * E).sum()).backward()
    api.stream_check()
    assert inputs.rel_fro(host(X.grad), oracle.correlation_vjp(d["X"], d["W"])) <= GATE
    G = 2.0 * host(E).astype(np.float64)
    for g, r in zip((A.grad, B.grad, C.grad), oracle.gemm_chain_vjp(d["A"], d["B"], d["C"], G)):
        assert inputs.rel_fro(host(g), r) <= GATE
