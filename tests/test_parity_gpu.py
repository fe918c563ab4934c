"""GPU parity: every kernel, form and precision against the FP64 oracle.

Gate (the relative Frobenius error of each output tensor against the exact
FP64 result): 1e-5 for FP32 (plain and tiled) and for the 3xBF16 / 6xBF16 /
3xTF32 split tensor-core modes; single-pass BF16 and TF32 are checked against a
loose sanity bound only. Integer-valued inputs must match bit for bit in every mode that
represents them exactly. Sizes span several tiles and ragged tails.
"""
import numpy as np
import pytest

import oracle
from paper_2312_13170_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = 1e-5
BF16_SANITY = 3e-2
MODES = [("plain", "fp32"), ("internalized", "fp32"), ("internalized", "bf16"),
         ("internalized", "3xbf16"), ("internalized", "6xbf16"), ("internalized", "tf32"),
         ("internalized", "3xtf32")]
LOOSE = ("bf16", "tf32")  # single-pass modes: a sanity bound, not the gate
EXACT_MODES = [m for m in MODES if m[1] not in LOOSE]
SINGLE_PASS = [("internalized", "bf16"), ("internalized", "tf32")]


def tol(prec):
    return BF16_SANITY if prec in LOOSE else GATE


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


# ------------------------------------------------------------------------ GEMM
@pytest.mark.parametrize("form,prec", MODES)
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (7, 33, 5), (129, 131, 67), (256, 256, 256), (300, 200, 513)])
def test_gemm(api, form, prec, M, N, K):
    d = inputs.gemm_inputs(M, N, K, seed=M + N + K)
    ref = oracle.gemm(d["A"], d["B"], d["C"], d["alpha"], d["beta"])
    C = dev(d["C"])
    api.gemm(dev(d["A"]), dev(d["B"]), C, d["alpha"], d["beta"], form=form, prec=prec)
    api.stream_check()
    assert inputs.rel_fro(host(C), ref) <= tol(prec)


def test_tf32_modes_are_tf32(api):
    """The TF32 modes round to TF32, not to BF16 or FP32: single-pass TF32's
    error sits between FP32's and BF16's, 3xTF32's below 3xBF16's."""
    d = inputs.gemm_inputs(512, 384, 640, seed=12)
    ref = oracle.gemm(d["A"], d["B"], d["C"], d["alpha"], d["beta"])
    err = {}
    for prec in ("bf16", "tf32", "3xbf16", "3xtf32", "fp32"):
        C = dev(d["C"])
        api.gemm(dev(d["A"]), dev(d["B"]), C, d["alpha"], d["beta"], prec=prec)
        err[prec] = inputs.rel_fro(host(C), ref)
    api.stream_check()
    assert err["fp32"] < err["tf32"] < err["bf16"] / 4, err
    assert err["3xtf32"] < err["3xbf16"] / 4 and err["3xtf32"] <= GATE, err
    assert 2e-5 < err["tf32"] < 3e-3, err


@pytest.mark.parametrize("form,prec", EXACT_MODES + SINGLE_PASS)
def test_gemm_integer_bitexact(api, form, prec):
    M, N, K = 150, 190, 300
    A, B, C = (inputs.int_matrix(s, seed=i) for i, s in enumerate([(M, K), (K, N), (M, N)]))
    ref = oracle.gemm(A, B, C, 2.0, -1.0)
    Ct = dev(C)
    api.gemm(dev(A), dev(B), Ct, 2.0, -1.0, form=form, prec=prec)
    assert np.array_equal(host(Ct).astype(np.float64), ref)


@pytest.mark.parametrize("form,prec", [("plain", "fp32"), ("internalized", "fp32"), ("internalized", "3xbf16"),
                                       ("internalized", "3xtf32")])
def test_gemm_edge_cases(api, form, prec):
    # K == 0: C = beta * C
    C = dev(inputs.gemm_inputs(5, 6, 1)["C"])
    C0 = host(C).copy()
    api.gemm(torch.empty((5, 0), device="cuda"), torch.empty((0, 6), device="cuda"), C, 1.5, 1.2, form=form, prec=prec)
    assert np.array_equal(host(C), (np.float32(1.2) * C0).astype(np.float32))
    # beta == 0: C is never read (NaN does not propagate)
    d = inputs.gemm_inputs(70, 40, 90, seed=3)
    Cn = torch.full((70, 40), float("nan"), device="cuda")
    api.gemm(dev(d["A"]), dev(d["B"]), Cn, 1.0, 0.0, form=form, prec=prec)
    assert inputs.rel_fro(host(Cn), oracle.gemm(d["A"], d["B"])) <= GATE
    # sub-matrix views with ld > columns and an odd (non-16-byte) base offset
    big = torch.from_numpy(inputs.gemm_inputs(200, 200, 200, seed=4)["A"]).cuda()
    A = big[1:101, 3:80]   # 100 x 77, ld 200, misaligned base
    B = big[5:82, 1:66]    # 77 x 65
    Cb = torch.zeros((120, 90), device="cuda")
    Cv = Cb[2:102, 1:66]
    api.gemm(A, B, Cv, 1.0, 0.0, form=form, prec=prec)
    ref = oracle.gemm(host(A), host(B))
    assert inputs.rel_fro(host(Cv), ref) <= GATE
    out = host(Cb)
    assert np.all(out[:2] == 0) and np.all(out[102:] == 0) and np.all(out[:, 66:] == 0) and np.all(out[:, :1] == 0)


def test_gemm_aliasing_rejected(api):
    A = torch.zeros((64, 64), device="cuda")
    with pytest.raises(api.LoopnestError) as e:
        api.gemm(A, torch.zeros((64, 64), device="cuda"), A, 1.0, 0.0)
    assert e.value.status == 2


# ------------------------------------------------------------------------ chain
@pytest.mark.parametrize("form,prec", MODES)
@pytest.mark.parametrize("ni,nj,nk,nl", [(1, 1, 1, 1), (65, 127, 33, 129), (200, 136, 264, 72), (256, 256, 256, 256)])
def test_chain(api, form, prec, ni, nj, nk, nl):
    d = inputs.chain_inputs(ni, nj, nk, nl, seed=ni + nl)
    E_ref, F_ref = oracle.gemm_chain(d["A"], d["B"], d["C"], d["D"], d["alpha"], d["beta"])
    E, F = api.gemm_chain(dev(d["A"]), dev(d["B"]), dev(d["C"]), dev(d["D"]), d["alpha"], d["beta"],
                          form=form, prec=prec)
    api.stream_check()
    assert inputs.rel_fro(host(E), E_ref) <= tol(prec)
    assert inputs.rel_fro(host(F), F_ref) <= tol(prec)


@pytest.mark.parametrize("form,prec", EXACT_MODES)
def test_chain_integer_bitexact(api, form, prec):
    ni, nj, nk, nl = 70, 64, 100, 90   # |T| <= 1600 (exact in two BF16 terms), |E| < 2^24
    A, B, C, D = (inputs.int_matrix(s, seed=10 + i) for i, s in enumerate([(ni, nk), (nk, nj), (nj, nl), (ni, nl)]))
    E_ref, F_ref = oracle.gemm_chain(A, B, C, D, 2.0, -1.0)
    E, F = api.gemm_chain(dev(A), dev(B), dev(C), dev(D), 2.0, -1.0, form=form, prec=prec)
    assert np.array_equal(host(E).astype(np.float64), E_ref)
    assert np.array_equal(host(F).astype(np.float64), F_ref)


# ------------------------------------------------------------------------ statistics, covariance, correlation
@pytest.mark.parametrize("form", ["plain", "internalized"])
@pytest.mark.parametrize("n,m", [(1, 5), (300, 131), (1000, 257)])
def test_col_stats(api, form, n, m):
    X = inputs.cov_inputs(n, m, seed=n)["X"]
    mean_ref, ss_ref = oracle.col_stats(X)
    mean, ss = api.col_stats(dev(X), form=form)
    assert np.max(np.abs(host(mean) - mean_ref) / np.maximum(np.abs(mean_ref), 1e-30)) < 1e-13
    if n > 1:
        assert np.max(np.abs(host(ss) - ss_ref) / ss_ref) < 1e-12


@pytest.mark.parametrize("form,prec", MODES)
@pytest.mark.parametrize("n,m", [(2, 1), (9, 7), (300, 131), (1000, 256)])
def test_covariance_correlation(api, form, prec, n, m):
    X = inputs.cov_inputs(n, m, seed=n + m)["X"]
    cov = api.covariance(dev(X), form=form, prec=prec)
    corr = api.correlation(dev(X), form=form, prec=prec)
    api.stream_check()
    cov_ref, corr_ref = oracle.covariance(X), oracle.correlation(X)
    c, r = host(cov), host(corr)
    assert inputs.rel_fro(c, cov_ref) <= tol(prec)
    assert inputs.rel_fro(r, corr_ref) <= tol(prec)
    assert np.array_equal(c, c.T) and np.array_equal(r, r.T)
    assert np.all(np.diag(r) == 1.0)
    if prec not in LOOSE:
        s = np.sqrt(np.diag(cov_ref))
        # error scaled by the columns' spreads: small-variance columns are checked too
        assert np.max(np.abs(c - cov_ref) / np.outer(s, s)) < 5e-5


@pytest.mark.parametrize("form,prec", EXACT_MODES)
def test_covariance_integer_bitexact(api, form, prec):
    n, m = 65, 40   # n - 1 = 64: the divisor is exact; integer column means make centring exact
    Z = inputs.int_matrix((n - 1, m), seed=5)
    X = np.concatenate([Z, -Z.sum(axis=0, keepdims=True)], axis=0) + np.arange(m, dtype=np.float32)[None, :] * 3
    X = X.astype(np.float32)
    ref = oracle.covariance(X)
    got = host(api.covariance(dev(X), form=form, prec=prec)).astype(np.float64)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("form,prec", [("plain", "fp32"), ("internalized", "fp32"), ("internalized", "3xbf16"),
                                       ("internalized", "3xtf32")])
def test_correlation_zero_variance_column(api, form, prec):
    X = inputs.cov_inputs(100, 6, seed=9)["X"]
    X[:, 2] = 42.0
    r = host(api.correlation(dev(X), form=form, prec=prec))
    assert np.all(r[2, [0, 1, 3, 4, 5]] == 0.0) and r[2, 2] == 1.0
    assert inputs.rel_fro(r, oracle.correlation(X)) <= GATE


# ------------------------------------------------------------------------ SYRK / SYR2K
@pytest.mark.parametrize("form,prec", MODES)
@pytest.mark.parametrize("fill", ["full", "lower", "upper"])
@pytest.mark.parametrize("n,k", [(1, 1), (33, 7), (130, 70), (257, 129)])
def test_syrk_syr2k(api, form, prec, fill, n, k):
    d = inputs.sym_inputs(n, k, seed=n * 3 + k)
    fl = {"full": 0, "lower": 1, "upper": 2}[fill]
    ref1 = oracle.syrk(d["A"], d["C"], d["alpha"], d["beta"], fl)
    ref2 = oracle.syr2k(d["A"], d["B"], d["C"], d["alpha"], d["beta"], fl)
    C1, C2 = dev(d["C"]), dev(d["C"])
    api.syrk(dev(d["A"]), C1, d["alpha"], d["beta"], fill=fill, form=form, prec=prec)
    api.syr2k(dev(d["A"]), dev(d["B"]), C2, d["alpha"], d["beta"], fill=fill, form=form, prec=prec)
    api.stream_check()
    g1, g2 = host(C1), host(C2)
    assert inputs.rel_fro(g1, ref1) <= tol(prec)
    assert inputs.rel_fro(g2, ref2) <= tol(prec)
    if fill != "full":  # the other triangle is untouched, bit for bit
        iu = np.triu_indices(n, 1) if fill == "lower" else np.tril_indices(n, -1)
        assert np.array_equal(g1[iu], d["C"][iu]) and np.array_equal(g2[iu], d["C"][iu])


@pytest.mark.parametrize("form,prec", EXACT_MODES + SINGLE_PASS)
def test_syrk_syr2k_integer_bitexact(api, form, prec):
    n, k = 140, 150
    A, B, C = inputs.int_matrix((n, k), seed=1), inputs.int_matrix((n, k), seed=2), inputs.int_matrix((n, n), seed=3)
    C = np.tril(C) + np.tril(C, -1).T
    C1, C2 = dev(C), dev(C)
    api.syrk(dev(A), C1, 2.0, -1.0, form=form, prec=prec)
    api.syr2k(dev(A), dev(B), C2, 2.0, -1.0, form=form, prec=prec)
    assert np.array_equal(host(C1).astype(np.float64), oracle.syrk(A, C, 2.0, -1.0))
    assert np.array_equal(host(C2).astype(np.float64), oracle.syr2k(A, B, C, 2.0, -1.0))


# ------------------------------------------------------------------------ batched
def _batch(count, lo, hi, seed):
    return inputs.sym_batch_inputs(count, lo, hi, seed=seed)


@pytest.mark.parametrize("form,prec", MODES)
@pytest.mark.parametrize("two", [False, True])
def test_batched(api, form, prec, two):
    b = _batch(9, 1, 300, seed=7)
    As = [dev(x["A"]) for x in b["instances"]]
    Bs = [dev(x["B"]) for x in b["instances"]] if two else None
    Cs = [dev(x["C"]) for x in b["instances"]]
    api.SymBatch(As, Cs, Bs, b["alpha"], b["beta"], form=form, prec=prec).run()
    api.stream_check()
    for x, C in zip(b["instances"], Cs):
        ref = (oracle.syr2k(x["A"], x["B"], x["C"], b["alpha"], b["beta"]) if two
               else oracle.syrk(x["A"], x["C"], b["alpha"], b["beta"]))
        assert inputs.rel_fro(host(C), ref) <= tol(prec), (x["n"], x["k"])


@pytest.mark.parametrize("form,prec", [("internalized", "fp32"), ("internalized", "3xbf16"),
                                       ("internalized", "3xtf32")])
def test_batched_single_instance_matches_unbatched(api, form, prec):
    d = inputs.sym_inputs(200, 90, seed=11)
    C1, C2 = dev(d["C"]), dev(d["C"])
    api.SymBatch([dev(d["A"])], [C1], [dev(d["B"])], 1.5, 1.2, form=form, prec=prec).run()
    api.syr2k(dev(d["A"]), dev(d["B"]), C2, 1.5, 1.2, form=form, prec=prec)
    assert np.array_equal(host(C1), host(C2))


def test_batched_graph_replay(api):
    """The device tile queue is reset inside the captured graph: two replays agree."""
    b = _batch(12, 16, 400, seed=3)
    As = [dev(x["A"]) for x in b["instances"]]
    Bs = [dev(x["B"]) for x in b["instances"]]
    Cs = [dev(x["C"]) for x in b["instances"]]
    C0 = [c.clone() for c in Cs]
    batch = api.SymBatch(As, Cs, Bs, b["alpha"], b["beta"], prec="3xbf16")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.run(s)  # warm-up outside capture (sets kernel attributes)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.run()
    outs = []
    for _ in range(2):
        for c, c0 in zip(Cs, C0):
            c.copy_(c0)
        g.replay()
        torch.cuda.synchronize()
        outs.append([host(c).copy() for c in Cs])
    for a, bb, x in zip(outs[0], outs[1], b["instances"]):
        assert np.array_equal(a, bb)
        assert inputs.rel_fro(a, oracle.syr2k(x["A"], x["B"], x["C"], b["alpha"], b["beta"])) <= GATE


# ------------------------------------------------------------------------ adjoints
@pytest.mark.parametrize("form,prec", [("plain", "fp32"), ("internalized", "fp32"), ("internalized", "3xbf16"),
                                       ("internalized", "3xtf32")])
def test_chain_bwd(api, form, prec):
    d = inputs.chain_inputs(96, 80, 112, 72, seed=2)
    G = inputs.gemm_inputs(96, 72, 1, seed=5)["C"]
    refs = oracle.gemm_chain_vjp(d["A"], d["B"], d["C"], G)
    got = api.gemm_chain_bwd(dev(d["A"]), dev(d["B"]), dev(d["C"]), dev(G), form=form, prec=prec)
    for g, r in zip(got, refs):
        assert inputs.rel_fro(host(g), r) <= GATE


@pytest.mark.parametrize("form,prec", [("plain", "fp32"), ("internalized", "fp32"), ("internalized", "3xbf16"),
                                       ("internalized", "3xtf32")])
@pytest.mark.parametrize("corr", [False, True])
def test_cov_corr_bwd(api, form, prec, corr):
    d = inputs.backward_inputs(300, 70, 8, seed=4)
    X, W = d["X"], d["W"][:70, :70].copy()
    ref = (oracle.correlation_vjp if corr else oracle.covariance_vjp)(X, W)
    fn = api.correlation_bwd if corr else api.covariance_bwd
    dX = fn(dev(X), dev(W), form=form, prec=prec)
    assert inputs.rel_fro(host(dX), ref) <= GATE
    mean, ss = api.col_stats(dev(X), form=form)
    dX2 = fn(dev(X), dev(W), stats=torch.cat([mean, ss]), form=form, prec=prec)
    assert inputs.rel_fro(host(dX2), ref) <= GATE


@pytest.mark.parametrize("form,prec", [("plain", "fp32"), ("internalized", "fp32"), ("internalized", "3xbf16"),
                                       ("internalized", "3xtf32")])
@pytest.mark.parametrize("corr", [False, True])
def test_cov_corr_fwd_keeps_stats(api, form, prec, corr):
    """ln_covariance_fwd / ln_correlation_fwd: the result bit for bit that of
    the plain call, the statistics bit for bit those of ln_col_stats, and the
    adjoint reading them equal to the one that recomputes them."""
    d = inputs.backward_inputs(333, 140, 8, seed=9)
    X, W = dev(d["X"]), dev(d["W"][:140, :140].copy())
    fwd, plain = (api.correlation_fwd, api.correlation) if corr else (api.covariance_fwd, api.covariance)
    out, stats = fwd(X, form=form, prec=prec)
    ref = plain(X, form=form, prec=prec)
    mean, ss = api.col_stats(X, form=form)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert torch.equal(stats, torch.cat([mean, ss]))
    assert inputs.rel_fro(host(out), (oracle.correlation if corr else oracle.covariance)(d["X"])) <= GATE
    bwd = api.correlation_bwd if corr else api.covariance_bwd
    dX1 = bwd(X, W, stats=stats, form=form, prec=prec)
    dX0 = bwd(X, W, form=form, prec=prec)
    torch.cuda.synchronize()
    assert torch.equal(dX1, dX0)


def test_autograd_functions(api):
    d = inputs.backward_inputs(256, 48, 40, seed=6)
    X = dev(d["X"]).requires_grad_(True)
    W = dev(d["W"][:48, :48].copy())
    A, B, C = (dev(d[k]).requires_grad_(True) for k in "ABC")
    R = api.CorrelationFn.apply(X, "internalized", "3xbf16", True)
    E = api.GemmChainFn.apply(A, B, C, "internalized", "3xbf16")
    L = (W * R).sum() + (E * E).sum()
    L.backward()
    Wn = d["W"][:48, :48]
    assert inputs.rel_fro(host(X.grad), oracle.correlation_vjp(d["X"], Wn)) <= GATE
    # upstream gradient of ||E||^2 is 2E, evaluated at the forward's own E
    G = 2.0 * host(E).astype(np.float64)
    for g, r in zip((A.grad, B.grad, C.grad), oracle.gemm_chain_vjp(d["A"], d["B"], d["C"], G)):
        assert inputs.rel_fro(host(g), r) <= GATE


# ------------------------------------------------------------------------ bounded waits
def test_bounded_wait_reports_timeout(api, monkeypatch):
    """A wait that nothing satisfies runs out, the kernel returns, the host
    reads LN_ERR_TIMEOUT, and the context stays usable."""
    d = inputs.gemm_inputs(128, 128, 128, seed=1)
    C = dev(d["C"])
    monkeypatch.setenv("LN_FAULT_INJECT", "timeout")
    api.gemm(dev(d["A"]), dev(d["B"]), C, 1.0, 0.0, prec="3xbf16")
    with pytest.raises(api.LoopnestError) as e:
        api.stream_check()
    assert e.value.status == 6
    monkeypatch.delenv("LN_FAULT_INJECT")
    api.gemm(dev(d["A"]), dev(d["B"]), C, 1.0, 0.0, prec="3xbf16")
    api.stream_check()
    assert inputs.rel_fro(host(C), oracle.gemm(d["A"], d["B"])) <= GATE
