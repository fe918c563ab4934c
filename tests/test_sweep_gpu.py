"""Seeded random shapes at tile boundaries, every operation, adjoint and form.

Each size is a multiple of 32, 64, 128 or 256 (one to three of them), or one
more or one less: the edges where the tcgen05 engine's 128-row and 64-k tiles,
its 128- and 256-wide column tiles, the FP32 form's 64- and 128-wide tiles
and the split-and-pack blocks start a ragged tile or an extra one. Each case
is drawn from its own seed, is checked once against the FP64 oracle, and then
runs in every form and precision that keeps the 1e-5 gate (single-pass BF16
and TF32 against a sanity bound).
"""
import zlib

import numpy as np
import pytest

import oracle
from paper_2312_13170_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = 1e-5
SANITY = 3e-2
MODES = [("plain", "fp32"), ("internalized", "fp32"), ("internalized", "bf16"), ("internalized", "3xbf16"),
         ("internalized", "6xbf16"), ("internalized", "tf32"), ("internalized", "3xtf32")]
CASES = 6


def tol(prec):
    return SANITY if prec in ("bf16", "tf32") else GATE


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


def draw(op, i, count):
    """`count` sizes for case i of `op`, and the case's seed."""
    seed = zlib.crc32(f"{op}/{i}".encode())
    rng = np.random.default_rng(seed)
    sizes = [int(rng.choice([32, 64, 128, 256])) * int(rng.integers(1, 4)) + int(rng.integers(-1, 2))
             for _ in range(count)]
    return sizes, seed


def check(got, ref, prec, what):
    err = inputs.rel_fro(got, ref)
    assert err <= tol(prec), f"{what} [{prec}]: relative error {err:.3e}"


@pytest.mark.parametrize("i", range(CASES))
def test_gemm_sweep(api, i):
    (M, N, K), seed = draw("gemm", i, 3)
    g = inputs.gemm_inputs(M, N, K, seed=seed)
    ref = oracle.gemm(g["A"], g["B"], g["C"], g["alpha"], g["beta"])
    A, B = dev(g["A"]), dev(g["B"])
    for form, prec in MODES:
        C = dev(g["C"])
        api.gemm(A, B, C, g["alpha"], g["beta"], form=form, prec=prec)
        check(host(C), ref, prec, f"gemm {M}x{N}x{K} {form}")
    api.stream_check()


@pytest.mark.parametrize("i", range(CASES))
def test_chain_sweep(api, i):
    (ni, nj, nk, nl), seed = draw("chain", i, 4)
    d = inputs.chain_inputs(ni, nj, nk, nl, seed=seed)
    E_ref, F_ref = oracle.gemm_chain(d["A"], d["B"], d["C"], d["D"], d["alpha"], d["beta"])
    t = {k: dev(d[k]) for k in "ABCD"}
    for form, prec in MODES:
        E, F = api.gemm_chain(t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], form=form, prec=prec)
        check(host(E), E_ref, prec, f"chain E {ni},{nj},{nk},{nl} {form}")
        check(host(F), F_ref, prec, f"chain F {ni},{nj},{nk},{nl} {form}")
    api.stream_check()


@pytest.mark.parametrize("i", range(CASES))
def test_3mm_sweep(api, i):
    (ni, nj, nk, nl, nm), seed = draw("3mm", i, 5)
    rng = np.random.default_rng(seed)
    A, B, C, D = (rng.uniform(-1, 1, size=s).astype(np.float32) for s in ((ni, nk), (nk, nj), (nj, nm), (nm, nl)))
    ref = oracle.three_mm(A, B, C, D)
    T = [dev(x) for x in (A, B, C, D)]
    for form, prec in MODES:
        G = api.three_mm(*T, form=form, prec=prec)
        check(host(G), ref, prec, f"3mm {ni},{nj},{nk},{nl},{nm} {form}")
    api.stream_check()


@pytest.mark.parametrize("i", range(CASES))
def test_syrk_syr2k_sweep(api, i):
    (n, k), seed = draw("sym", i, 2)
    fill = ("full", "lower", "upper")[seed % 3]
    fl = {"full": 0, "lower": 1, "upper": 2}[fill]
    d = inputs.sym_inputs(n, k, seed=seed)
    r1 = oracle.syrk(d["A"], d["C"], d["alpha"], d["beta"], fl)
    r2 = oracle.syr2k(d["A"], d["B"], d["C"], d["alpha"], d["beta"], fl)
    A, B = dev(d["A"]), dev(d["B"])
    keep = None if fill == "full" else (np.triu_indices(n, 1) if fill == "lower" else np.tril_indices(n, -1))
    for form, prec in MODES:
        C1, C2 = dev(d["C"]), dev(d["C"])
        api.syrk(A, C1, d["alpha"], d["beta"], fill=fill, form=form, prec=prec)
        api.syr2k(A, B, C2, d["alpha"], d["beta"], fill=fill, form=form, prec=prec)
        c1, c2 = host(C1), host(C2)
        check(c1, r1, prec, f"syrk n={n} k={k} {fill} {form}")
        check(c2, r2, prec, f"syr2k n={n} k={k} {fill} {form}")
        if keep is not None:  # the other triangle is not touched
            assert np.array_equal(c1[keep], d["C"][keep]) and np.array_equal(c2[keep], d["C"][keep])
    api.stream_check()


@pytest.mark.parametrize("i", range(CASES))
def test_cov_corr_sweep(api, i):
    (n, m), seed = draw("cov", i, 2)
    X = inputs.cov_inputs(n, m, seed=seed)["X"]
    cov_ref, corr_ref = oracle.covariance(X), oracle.correlation(X)
    Xd = dev(X)
    for form, prec in MODES:
        cov = host(api.covariance(Xd, form=form, prec=prec))
        corr = host(api.correlation(Xd, form=form, prec=prec))
        check(cov, cov_ref, prec, f"covariance {n}x{m} {form}")
        check(corr, corr_ref, prec, f"correlation {n}x{m} {form}")
        assert np.array_equal(cov, cov.T) and np.array_equal(corr, corr.T)
    api.stream_check()


# adjoints: the forms and precisions that keep the gate
EXACT = [m for m in MODES if m[1] not in ("bf16", "tf32")]


@pytest.mark.parametrize("i", range(CASES))
def test_chain_bwd_sweep(api, i):
    (ni, nj, nk, nl), seed = draw("chain_bwd", i, 4)
    d = inputs.chain_inputs(ni, nj, nk, nl, seed=seed)
    G = inputs.gemm_inputs(ni, nl, 1, seed=seed + 1)["C"]
    refs = oracle.gemm_chain_vjp(d["A"], d["B"], d["C"], G)
    t = [dev(x) for x in (d["A"], d["B"], d["C"], G)]
    for form, prec in EXACT:
        got = api.gemm_chain_bwd(*t, form=form, prec=prec)
        for name, g, r in zip(("dA", "dB", "dC"), got, refs):
            check(host(g), r, prec, f"chain {name} {ni},{nj},{nk},{nl} {form}")
    api.stream_check()


@pytest.mark.parametrize("i", range(CASES))
def test_3mm_bwd_sweep(api, i):
    (ni, nj, nk, nl, nm), seed = draw("3mm_bwd", i, 5)
    rng = np.random.default_rng(seed)
    mats = [rng.uniform(-1, 1, size=s).astype(np.float32)
            for s in ((ni, nk), (nk, nj), (nj, nm), (nm, nl), (ni, nl))]
    refs = oracle.three_mm_vjp(*mats)
    t = [dev(x) for x in mats]
    for form, prec in EXACT:
        got = api.three_mm_bwd(*t, form=form, prec=prec)
        for name, g, r in zip(("dA", "dB", "dC", "dD"), got, refs):
            check(host(g), r, prec, f"3mm {name} {ni},{nj},{nk},{nl},{nm} {form}")
    api.stream_check()


@pytest.mark.parametrize("i", range(CASES))
def test_cov_corr_bwd_sweep(api, i):
    (n, m), seed = draw("cov_bwd", i, 2)
    X = inputs.cov_inputs(n, m, seed=seed)["X"]
    W = np.random.default_rng(seed).uniform(-1, 1, size=(m, m)).astype(np.float32)
    rc, rr = oracle.covariance_vjp(X, W), oracle.correlation_vjp(X, W)
    Xd, Wd = dev(X), dev(W)
    for form, prec in EXACT:
        check(host(api.covariance_bwd(Xd, Wd, form=form, prec=prec)), rc, prec, f"covariance dX {n}x{m} {form}")
        check(host(api.correlation_bwd(Xd, Wd, form=form, prec=prec)), rr, prec, f"correlation dX {n}x{m} {form}")
    api.stream_check()


@pytest.mark.parametrize("i", range(CASES))
@pytest.mark.parametrize("two", [False, True])
def test_batched_sweep(api, i, two):
    """One batch of 24 instances whose n and k are drawn at tile edges, in one
    fill, through the persistent batched kernel (SymBatch)."""
    sizes, seed = draw("batched", i, 48)
    fill = ("full", "lower", "upper")[seed % 3]
    fl = {"full": 0, "lower": 1, "upper": 2}[fill]
    inst = [inputs.sym_inputs(n, k, seed=seed + j) for j, (n, k) in enumerate(zip(sizes[0::2], sizes[1::2]))]
    alpha, beta = inst[0]["alpha"], inst[0]["beta"]
    refs = [oracle.syr2k(x["A"], x["B"], x["C"], alpha, beta, fl) if two else
            oracle.syrk(x["A"], x["C"], alpha, beta, fl) for x in inst]
    As = [dev(x["A"]) for x in inst]
    Bs = [dev(x["B"]) for x in inst] if two else None
    for form, prec in MODES:
        Cs = [dev(x["C"]) for x in inst]
        api.SymBatch(As, Cs, Bs, alpha, beta, fill=fill, form=form, prec=prec).run()
        api.stream_check()
        for x, C, r in zip(inst, Cs, refs):
            check(host(C), r, prec, f"batched {'syr2k' if two else 'syrk'} n={x['A'].shape[0]} "
                                    f"k={x['A'].shape[1]} {fill} {form}")


@pytest.mark.parametrize("i", range(CASES))
def test_gramschmidt_sweep(api, i):
    """Modified Gram-Schmidt QR of an m x n matrix (m >= n) drawn at tile
    edges: R within the gate, Q within the gate or the conditioning bound, QR
    reproducing A, R upper triangular with a non-negative diagonal."""
    sizes, seed = draw("gramschmidt", i, 2)
    m, n = max(sizes), min(sizes)
    A = inputs.gramschmidt_inputs(m, n, seed=seed)["A"]
    Qo, Ro = oracle.gramschmidt(A)
    kappa = np.linalg.cond(A.astype(np.float64))
    for form in ("plain", "internalized"):
        Q, R = api.gramschmidt(dev(A), form=form)
        api.stream_check()
        Q, R = host(Q), host(R)
        assert np.array_equal(np.tril(R, -1), np.zeros_like(R)) and np.all(np.diag(R) >= 0), (m, n, form)
        assert inputs.rel_fro(R, Ro) <= GATE, (m, n, form)
        assert inputs.rel_fro(Q, Qo) <= max(GATE, kappa * 2.0 ** -24), (m, n, form)
        assert inputs.rel_fro(Q @ R, A.astype(np.float64)) <= GATE, (m, n, form)
