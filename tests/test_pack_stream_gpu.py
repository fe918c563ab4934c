"""GPU parity of the split-and-pack paths, bit for bit on integer inputs.

The split-and-pack stage has three paths: the bulk-copy stream (sources with
16-byte-aligned rows of whole 16-byte units), the element-wise fallback, and
the stream run by the spare CTAs of the chain's first contraction (the chain
packs C there when the first product has fewer output tiles than SMs, and
separately otherwise). Integer-valued inputs make every split product and
partial sum exact, so each path must reproduce the FP64 oracle exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2312_13170_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("prec", ["3xbf16", "6xbf16"])
@pytest.mark.parametrize("ni,nj,nk,nl", [
    (200, 136, 264, 92),    # stream for A, B; C on the spare CTAs of the first product
    (2560, 2048, 64, 64),   # 160 output tiles >= SMs: no spare CTAs, C packed after the first product
    (150, 130, 99, 90),     # K of A and rows of C not multiples of 4: element-wise fallback
    (129, 257, 65, 131),    # ragged tiles everywhere
])
def test_chain_pack_paths_bitexact(api, prec, ni, nj, nk, nl):
    # |T| <= 16 nk (exact in two BF16 terms), |E| <= 64 nk nj < 2^24
    A, B, C, D = (inputs.int_matrix(s, seed=20 + i) for i, s in enumerate([(ni, nk), (nk, nj), (nj, nl), (ni, nl)]))
    E_ref, F_ref = oracle.gemm_chain(A, B, C, D, 2.0, -1.0)
    E, F = api.gemm_chain(dev(A), dev(B), dev(C), dev(D), 2.0, -1.0, prec=prec)
    api.stream_check()
    assert np.array_equal(host(E).astype(np.float64), E_ref)
    assert np.array_equal(host(F).astype(np.float64), F_ref)


@pytest.mark.parametrize("prec", ["bf16", "3xbf16", "6xbf16"])
@pytest.mark.parametrize("M,N,K", [(300, 260, 388), (300, 260, 387), (128, 256, 64), (5, 4, 4)])
def test_gemm_pack_paths_bitexact(api, prec, M, N, K):
    A, B, C = (inputs.int_matrix(s, seed=30 + i) for i, s in enumerate([(M, K), (K, N), (M, N)]))
    ref = oracle.gemm(A, B, C, 2.0, -1.0)
    Ct = dev(C)
    api.gemm(dev(A), dev(B), Ct, 2.0, -1.0, prec=prec)
    api.stream_check()
    assert np.array_equal(host(Ct).astype(np.float64), ref)


@pytest.mark.parametrize("prec", ["3xbf16", "6xbf16"])
@pytest.mark.parametrize("n,m", [(500, 132), (300, 131)])
def test_covariance_pack_paths_bitexact(api, prec, n, m):
    # X = [Y; -Y] + 1 c^T with small integers: every column mean is the integer
    # c_j, the centred values are +-Y (exact in one BF16 term) and the sums of
    # products are integers below 2^24, so the only rounding is the final
    # scaling by 1/(n-1) (at most 2 units in the last place of FP32)
    Y = inputs.int_matrix((n // 2, m), lo=-8, hi=8, seed=40)
    c = inputs.int_matrix((1, m), lo=-50, hi=50, seed=41)
    X = (np.concatenate([Y, -Y]) + c).astype(np.float32)
    ref = oracle.covariance(X)
    got = host(api.covariance(dev(X), prec=prec)).astype(np.float64)
    assert np.all(np.abs(got - ref) <= 2.5e-7 * np.abs(ref))


def test_chain_fullsize_side_pack_matches_separate(api):
    """The 2048 chain (128 output tiles) packs C on the spare CTAs; its result
    equals the same chain computed with C packed up front (tile width 128:
    256 tiles, no spare CTAs) up to the summation order of the tile widths."""
    d = inputs.chain_inputs(2048, seed=0)
    t = {k: dev(d[k]) for k in "ABCD"}
    E1, F1 = api.gemm_chain(t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], prec="3xbf16")
    api.set_tuning("tile_n", 128)
    try:
        E2, F2 = api.gemm_chain(t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], prec="3xbf16")
    finally:
        api.set_tuning("tile_n", 0)
    api.stream_check()
    rows = np.arange(0, 2048, 97)
    E_ref, F_ref = oracle.gemm_chain(d["A"][rows], d["B"], d["C"], d["D"][rows], d["alpha"], d["beta"])
    for E in (E1, E2):
        assert inputs.rel_fro(host(E)[rows], E_ref) <= 1e-5
    assert inputs.rel_fro(host(F1), host(F2)) <= 2e-6


@pytest.mark.parametrize("prec", ["3xbf16", "6xbf16"])
def test_split_k_graph_replay(api, prec):
    """Few output tiles and a long reduction: the contraction is split along K
    (slices hand partial sums to the last arrival through the workspace, with
    arrival counters zeroed per call), so replaying a captured call repeats
    the same result bit for bit."""
    api.set_tuning("split_k", 1)
    try:
        _split_k_graph_replay(api, prec)
    finally:
        api.set_tuning("split_k", 0)


def _split_k_graph_replay(api, prec):
    A, B = (inputs.int_matrix(s, seed=50 + i) for i, s in enumerate([(1024, 1024), (1024, 1024)]))
    ref = oracle.gemm(A, B)
    At, Bt = dev(A), dev(B)
    C = torch.empty((1024, 1024), device="cuda")
    api.gemm(At, Bt, C, 1.0, 0.0, prec=prec)  # warm (workspace, attributes)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        api.gemm(At, Bt, C, 1.0, 0.0, prec=prec)
    for _ in range(3):
        C.fill_(float("nan"))
        g.replay()
        api.stream_check()
        assert np.array_equal(host(C).astype(np.float64), ref)


@pytest.mark.parametrize("prec", ["3xbf16", "6xbf16"])
def test_split_k_parity(api, prec):
    """With split-K on: general, chain, symmetric and backward contractions with
    few output tiles against the oracle (integer inputs: bit for bit)."""
    api.set_tuning("split_k", 1)
    try:
        M, N, K = 300, 260, 2000
        A, B, C = (inputs.int_matrix(s, seed=60 + i) for i, s in enumerate([(M, K), (K, N), (M, N)]))
        Ct = dev(C)
        api.gemm(dev(A), dev(B), Ct, 2.0, -1.0, prec=prec)
        assert np.array_equal(host(Ct).astype(np.float64), oracle.gemm(A, B, C, 2.0, -1.0))
        ni, nj, nk, nl = 200, 136, 1000, 92
        A, B, Cc, D = (inputs.int_matrix(s, seed=70 + i) for i, s in enumerate([(ni, nk), (nk, nj), (nj, nl), (ni, nl)]))
        E_ref, F_ref = oracle.gemm_chain(A, B, Cc, D, 2.0, -1.0)
        E, F = api.gemm_chain(dev(A), dev(B), dev(Cc), dev(D), 2.0, -1.0, prec=prec)
        assert np.array_equal(host(E).astype(np.float64), E_ref)
        assert np.array_equal(host(F).astype(np.float64), F_ref)
        n, k = 260, 1500
        A, Cs = inputs.int_matrix((n, k), seed=80), inputs.int_matrix((n, n), seed=81)
        Cs = (Cs + Cs.T).astype(np.float32)
        Ct = dev(Cs)
        api.syrk(dev(A), Ct, 2.0, -1.0, prec=prec)
        assert np.array_equal(host(Ct).astype(np.float64), oracle.syrk(A, Cs, 2.0, -1.0))
        d = inputs.backward_inputs(256, 16, 1024, seed=3)
        t = {k: dev(d[k]) for k in ("A", "B", "C")}
        G = dev(d["A"])
        dA, dB, dC = api.gemm_chain_bwd(t["A"], t["B"], t["C"], G, prec=prec)
        rA, rB, rC = oracle.gemm_chain_vjp(d["A"], d["B"], d["C"], d["A"])
        for got, ref in ((dA, rA), (dB, rB), (dC, rC)):
            assert inputs.rel_fro(host(got), ref) <= 1e-5
        api.stream_check()
    finally:
        api.set_tuning("split_k", 0)


@pytest.mark.parametrize("prec", ["fp32", "3xbf16"])
def test_chain_host_resident_operands(api, prec):
    """Pinned host operands and outputs: the kernels read A..D and write E, F in
    host memory directly; the result equals the device-resident call bit for
    bit, and pageable host tensors are refused by the binding."""
    form = "internalized"
    d = inputs.chain_inputs(520, 264, 300, 392, seed=9)
    host = {k: torch.from_numpy(d[k]).pin_memory() for k in "ABCD"}
    devt = {k: v.cuda() for k, v in host.items()}
    E, F = api.gemm_chain(devt["A"], devt["B"], devt["C"], devt["D"], d["alpha"], d["beta"], form=form, prec=prec)
    hE = torch.empty(E.shape).pin_memory()
    hF = torch.empty(E.shape).pin_memory()
    api.gemm_chain(host["A"], host["B"], host["C"], host["D"], d["alpha"], d["beta"], form=form, prec=prec,
                   out=(hE, hF))
    api.stream_check()
    assert torch.equal(hE, E.cpu()) and torch.equal(hF, F.cpu())
    with pytest.raises(TypeError):
        api.gemm_chain(torch.from_numpy(d["A"]), host["B"], host["C"], host["D"], 1.0, 1.0, prec=prec)
