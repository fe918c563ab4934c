"""CTA pairs of the tensor-core contractions (the "pair" knob: 1, the default,
pairs 256-wide general tiles of the split precisions, BF16 and TF32 operands;
2, used here, also single-pass BF16 and TF32, and every width with BF16
operands, symmetric outputs included).

Two CTAs of a cluster compute vertically adjacent output tiles and each copies
half of the shared column operand into both CTAs' shared memory. Every tile is
computed from the same operands in the same order as without pairs, so the
results must be bit-identical to the unpaired launch, and within the 1e-5 gate
of the FP64 oracle. The sizes cover an odd number of row tiles (the last pair's
second CTA has no tile), symmetric outputs (the pair tile above the diagonal),
ragged edges, all fills, batched-free single problems and CUDA graph replay.
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

    yield a
    a.set_tuning("pair", 1)


ON = 2  # every tile width


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def paired_and_not(api, fn):
    out = []
    for on in (ON, 0):
        api.set_tuning("pair", on)
        out.append(fn())
        api.stream_check()
    api.set_tuning("pair", 1)
    return out


@pytest.mark.parametrize("prec", ["bf16", "3xbf16", "6xbf16", "tf32", "3xtf32"])
@pytest.mark.parametrize("M,N,K", [(300, 517, 389), (256, 256, 256), (1000, 1100, 700), (129, 77, 1000)])
def test_gemm_pairs(api, prec, M, N, K):
    g = inputs.gemm_inputs(M, N, K, seed=M + N)

    def run():
        C = dev(g["C"])
        api.gemm(dev(g["A"]), dev(g["B"]), C, g["alpha"], g["beta"], prec=prec)
        return host(C)

    on, off = paired_and_not(api, run)
    assert np.array_equal(on, off)
    if prec not in ("bf16", "tf32"):
        assert inputs.rel_fro(on, oracle.gemm(g["A"], g["B"], g["C"], g["alpha"], g["beta"])) <= GATE


def test_gemm_pairs_integer_bitexact(api):
    A, B, C = inputs.int_matrix((700, 900), seed=1), inputs.int_matrix((900, 650), seed=2), inputs.int_matrix(
        (700, 650), seed=3)
    Cd = dev(C)
    api.gemm(dev(A), dev(B), Cd, 2.0, -1.0, prec="3xbf16")
    assert np.array_equal(host(Cd).astype(np.float64), oracle.gemm(A, B, C, 2.0, -1.0))


@pytest.mark.parametrize("prec", ["3xbf16", "3xtf32"])
@pytest.mark.parametrize("shape", [(2048, 2048, 2048, 2048), (333, 257, 500, 129), (1500, 700, 900, 1300)])
def test_chain_pairs(api, shape, prec):
    d = inputs.chain_inputs(*shape, seed=41)
    t = {k: dev(d[k]) for k in "ABCD"}

    def run():
        E, F = api.gemm_chain(t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], prec=prec)
        return host(E), host(F)

    (E1, F1), (E0, F0) = paired_and_not(api, run)
    assert np.array_equal(E1, E0) and np.array_equal(F1, F0)
    rows = slice(0, 64)
    E_ref, F_ref = oracle.gemm_chain(d["A"][rows], d["B"], d["C"], d["D"][rows], d["alpha"], d["beta"])
    assert inputs.rel_fro(E1[rows], E_ref) <= GATE and inputs.rel_fro(F1[rows], F_ref) <= GATE


@pytest.mark.parametrize("prec", ["3xbf16", "3xtf32"])
def test_3mm_pairs(api, prec):
    rng = np.random.default_rng(42)
    A, B, C, D = (rng.uniform(-1, 1, size=s).astype(np.float32) for s in ((700, 500), (500, 900), (900, 300),
                                                                          (300, 650)))
    T = [dev(x) for x in (A, B, C, D)]
    on, off = paired_and_not(api, lambda: host(api.three_mm(*T, prec=prec)))
    assert np.array_equal(on, off)
    assert inputs.rel_fro(on, oracle.three_mm(A, B, C, D)) <= GATE


@pytest.mark.parametrize("fill", ["full", "lower", "upper"])
@pytest.mark.parametrize("n,k", [(257, 129), (640, 300), (1500, 700)])
def test_syrk_syr2k_pairs(api, fill, n, k):
    d = inputs.sym_inputs(n, k, seed=n + k)
    fl = {"full": 0, "lower": 1, "upper": 2}[fill]

    def run():
        C1, C2 = dev(d["C"]), dev(d["C"])
        api.syrk(dev(d["A"]), C1, d["alpha"], d["beta"], fill=fill, prec="3xbf16")
        api.syr2k(dev(d["A"]), dev(d["B"]), C2, d["alpha"], d["beta"], fill=fill, prec="3xbf16")
        return host(C1), host(C2)

    (a1, a2), (b1, b2) = paired_and_not(api, run)
    assert np.array_equal(a1, b1) and np.array_equal(a2, b2)
    assert inputs.rel_fro(a1, oracle.syrk(d["A"], d["C"], d["alpha"], d["beta"], fl)) <= GATE
    assert inputs.rel_fro(a2, oracle.syr2k(d["A"], d["B"], d["C"], d["alpha"], d["beta"], fl)) <= GATE
    if fill != "full":
        iu = np.triu_indices(n, 1) if fill == "lower" else np.tril_indices(n, -1)
        assert np.array_equal(a1[iu], d["C"][iu]) and np.array_equal(a2[iu], d["C"][iu])


@pytest.mark.parametrize("n,m", [(1000, 300), (8192, 2048)])
def test_cov_corr_pairs(api, n, m):
    X = inputs.cov_inputs(n, m, seed=n + m + 3)["X"]
    Xd = dev(X)
    (c1, r1), (c0, r0) = paired_and_not(api, lambda: (host(api.covariance(Xd, prec="3xbf16")),
                                                       host(api.correlation(Xd, prec="3xbf16"))))
    assert np.array_equal(c1, c0) and np.array_equal(r1, r0)
    rows = [0, 1, m // 2, m - 1]
    assert inputs.rel_fro(c1[rows], oracle.cov_rows(X, rows)) <= GATE
    assert inputs.rel_fro(r1[rows], oracle.cov_rows(X, rows, corr=True)) <= GATE
    assert np.array_equal(c1, c1.T) and np.all(np.diag(r1) == 1.0)


def test_pairs_graph_replay(api):
    d = inputs.chain_inputs(640, 512, 384, 768, seed=43)
    t = {k: dev(d[k]) for k in "ABCD"}
    E = torch.empty((640, 768), device="cuda")
    F = torch.empty_like(E)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        api.gemm_chain(t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], prec="3xbf16", out=(E, F), stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        api.gemm_chain(t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], prec="3xbf16", out=(E, F))
    outs = []
    for _ in range(2):
        E.fill_(float("nan"))
        g.replay()
        outs.append(host(E))
    api.stream_check()
    assert np.array_equal(outs[0], outs[1])
    E_ref, _ = oracle.gemm_chain(d["A"], d["B"], d["C"], d["D"], d["alpha"], d["beta"])
    assert inputs.rel_fro(outs[0], E_ref) <= GATE


@pytest.mark.parametrize("shape", [(2048, 2048, 2048, 2048), (1000, 700, 1300, 1100)])
def test_stage_beta_bit_identical(api, shape):
    """Staging the last tile's block of D (chain) or C (GEMM) in shared memory
    changes where the epilogue reads it from, not the result."""
    d = inputs.chain_inputs(*shape, seed=44)
    t = {k: dev(d[k]) for k in "ABCD"}
    g = inputs.gemm_inputs(1000, 1100, 700, seed=45)
    out = []
    for on in (1, 0):
        api.set_tuning("stage_beta", on)
        E, F = api.gemm_chain(t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], prec="3xbf16")
        C = dev(g["C"])
        api.gemm(dev(g["A"]), dev(g["B"]), C, g["alpha"], g["beta"], prec="3xbf16")
        out.append((host(E), host(F), host(C)))
    api.set_tuning("stage_beta", 1)
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    rows = slice(0, 48)
    E_ref, F_ref = oracle.gemm_chain(d["A"][rows], d["B"], d["C"], d["D"][rows], d["alpha"], d["beta"])
    assert inputs.rel_fro(out[0][1][rows], F_ref) <= GATE
    assert inputs.rel_fro(out[0][2], oracle.gemm(g["A"], g["B"], g["C"], g["alpha"], g["beta"])) <= GATE


@pytest.mark.parametrize("shape", [(2048, 2048, 2048, 2048), (1500, 1700, 900, 1100)])
@pytest.mark.parametrize("pair", [0, 1])
def test_stage_out_bit_identical(api, shape, pair):
    """Building the packed intermediate (the chain's T, 3mm's E and F) of a
    CTA's last 256-wide tile in the freed stage memory and bulk-storing it
    changes how it reaches global memory, not the result. The second shape has
    ragged row and column tiles; both take 256-wide tiles."""
    d = inputs.chain_inputs(*shape, seed=46)
    t = {k: dev(d[k]) for k in "ABCD"}
    rng = np.random.default_rng(47)
    ni, nj = shape[0], shape[1]
    m3 = [rng.uniform(-1, 1, size=s).astype(np.float32) for s in ((ni, 600), (600, nj), (nj, 500), (500, 1100))]
    t3 = [dev(x) for x in m3]
    out = []
    api.set_tuning("pair", pair)
    try:
        for on in (1, 0):
            api.set_tuning("stage_out", on)
            E, F = api.gemm_chain(t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], prec="3xbf16")
            G = api.three_mm(*t3, prec="3xbf16")
            api.stream_check()
            out.append((host(E), host(F), host(G)))
    finally:
        api.set_tuning("stage_out", 1)
        api.set_tuning("pair", 1)
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    rows = slice(0, 40)
    E_ref, F_ref = oracle.gemm_chain(d["A"][rows], d["B"], d["C"], d["D"][rows], d["alpha"], d["beta"])
    assert inputs.rel_fro(out[0][0][rows], E_ref) <= GATE and inputs.rel_fro(out[0][1][rows], F_ref) <= GATE
    G_ref = oracle.three_mm(m3[0][rows], m3[1], m3[2], m3[3])
    assert inputs.rel_fro(out[0][2][rows], G_ref) <= GATE
