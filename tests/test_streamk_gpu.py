"""Stream-K decomposition of the tensor-core contractions (the "stream_k" knob).

When a contraction has fewer output tiles than SMs, its tiles x k-tiles units
are split evenly over one CTA per SM; tiles whose k range spans several CTAs
exchange FP32 partial sums through the workspace and are finished, in k order,
by the CTA holding the first k tile. These sizes all take that path (ragged
edges included) and are checked against the FP64 oracle within the 1e-5 gate,
bit for bit on integer inputs, against the same call without stream-K, and
under CUDA graph replay (the flags are cleared inside the captured call).
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
    a.set_tuning("stream_k", 2)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def both(api, fn):
    """fn() with stream-K on, then off."""
    out = []
    for on in (1, 0):
        api.set_tuning("stream_k", on)
        out.append(fn())
        api.stream_check()
    api.set_tuning("stream_k", 2)
    return out


@pytest.mark.parametrize("prec", ["3xbf16", "6xbf16"])
def test_gemm_streamk(api, prec):
    g = inputs.gemm_inputs(1000, 1100, 1300, seed=31)
    ref = oracle.gemm(g["A"], g["B"], g["C"], g["alpha"], g["beta"])

    def run():
        C = dev(g["C"])
        api.gemm(dev(g["A"]), dev(g["B"]), C, g["alpha"], g["beta"], prec=prec)
        return host(C)

    on, off = both(api, run)
    assert inputs.rel_fro(on, ref) <= GATE and inputs.rel_fro(off, ref) <= GATE


@pytest.mark.parametrize("prec", ["3xbf16", "6xbf16", "bf16"])
def test_gemm_streamk_integer_bitexact(api, prec):
    A, B = inputs.int_matrix((700, 1500), seed=1), inputs.int_matrix((1500, 900), seed=2)
    C = inputs.int_matrix((700, 900), seed=3)
    ref = oracle.gemm(A, B, C, 2.0, -1.0)

    def run():
        Cd = dev(C)
        api.gemm(dev(A), dev(B), Cd, 2.0, -1.0, prec=prec)
        return host(Cd)

    on, off = both(api, run)
    assert np.array_equal(on.astype(np.float64), ref) and np.array_equal(off, on)


def test_chain_streamk(api):
    d = inputs.chain_inputs(1000, 1024, 1100, 900, seed=32)
    E_ref, F_ref = oracle.gemm_chain(d["A"], d["B"], d["C"], d["D"], d["alpha"], d["beta"])
    t = {k: dev(d[k]) for k in "ABCD"}

    def run():
        E, F = api.gemm_chain(t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], prec="3xbf16")
        return host(E), host(F)

    (E1, F1), (E0, F0) = both(api, run)
    for E, F in ((E1, F1), (E0, F0)):
        assert inputs.rel_fro(E, E_ref) <= GATE and inputs.rel_fro(F, F_ref) <= GATE


def test_chain_streamk_integer_bitexact(api):
    n = 1024
    A, B, C, D = (inputs.int_matrix((n, n), lo=-2, hi=2, seed=s) for s in (4, 5, 6, 7))
    B = (B * (np.abs(B) < 2)).astype(np.float32)  # T stays a small integer matrix (exact as split BF16 terms)
    E_ref, F_ref = oracle.gemm_chain(A, B, C, D, 2.0, -1.0)
    assert np.max(np.abs(E_ref)) < 2 ** 24

    def run():
        E, F = api.gemm_chain(dev(A), dev(B), dev(C), dev(D), 2.0, -1.0, prec="3xbf16")
        return host(E), host(F)

    (E1, F1), (E0, F0) = both(api, run)
    assert np.array_equal(E1.astype(np.float64), E_ref) and np.array_equal(F1.astype(np.float64), F_ref)
    assert np.array_equal(E0, E1) and np.array_equal(F0, F1)


def test_3mm_streamk(api):
    rng = np.random.default_rng(33)
    A, B, C, D = (rng.uniform(-1, 1, size=s).astype(np.float32) for s in ((1400, 1300), (1300, 1500), (1500, 1200),
                                                                          (1200, 1100)))
    ref = oracle.three_mm(A, B, C, D)
    T = [dev(x) for x in (A, B, C, D)]
    on, off = both(api, lambda: host(api.three_mm(*T, prec="3xbf16")))
    assert inputs.rel_fro(on, ref) <= GATE and inputs.rel_fro(off, ref) <= GATE


@pytest.mark.parametrize("fill", ["full", "lower", "upper"])
def test_syrk_syr2k_streamk(api, fill):
    d = inputs.sym_inputs(1500, 700, seed=34)
    fl = {"full": 0, "lower": 1, "upper": 2}[fill]
    ref1 = oracle.syrk(d["A"], d["C"], d["alpha"], d["beta"], fl)
    ref2 = oracle.syr2k(d["A"], d["B"], d["C"], d["alpha"], d["beta"], fl)

    def run():
        C1, C2 = dev(d["C"]), dev(d["C"])
        api.syrk(dev(d["A"]), C1, d["alpha"], d["beta"], fill=fill, prec="3xbf16")
        api.syr2k(dev(d["A"]), dev(d["B"]), C2, d["alpha"], d["beta"], fill=fill, prec="3xbf16")
        return host(C1), host(C2)

    (g1, g2), (h1, h2) = both(api, run)
    for a, b in ((g1, g2), (h1, h2)):
        assert inputs.rel_fro(a, ref1) <= GATE and inputs.rel_fro(b, ref2) <= GATE
    if fill != "full":
        iu = np.triu_indices(1500, 1) if fill == "lower" else np.tril_indices(1500, -1)
        assert np.array_equal(g1[iu], d["C"][iu]) and np.array_equal(g2[iu], d["C"][iu])


def test_cov_corr_streamk(api):
    X = inputs.cov_inputs(3000, 1200, seed=35)["X"]
    cov_ref, corr_ref = oracle.covariance(X), oracle.correlation(X)
    Xd = dev(X)
    (c1, r1), (c0, r0) = both(api, lambda: (host(api.covariance(Xd, prec="3xbf16")),
                                             host(api.correlation(Xd, prec="3xbf16"))))
    for c, r in ((c1, r1), (c0, r0)):
        assert inputs.rel_fro(c, cov_ref) <= GATE and inputs.rel_fro(r, corr_ref) <= GATE
        assert np.array_equal(c, c.T) and np.all(np.diag(r) == 1.0)


def test_streamk_automatic_policy(api):
    """The default (2) takes stream-K only for deep contractions filling at
    most half the SMs: the correlation of a 4096 x 1024 matrix (36 tiles of 64
    k tiles; its workspace grows by the partial-sum area) but not the
    8192 x 2048 covariance (136 tiles). Results: oracle gate, and integer SYRK
    of the same shape bit for bit against stream-K off."""
    import ctypes

    assert api.get_tuning("stream_k") == 2

    def ws(n, m):
        b = ctypes.c_size_t()
        assert api.lib().ln_covariance_workspace_size(n, m, 1, 2, ctypes.byref(b)) == 0
        return b.value

    sizes = {}
    for v in (0, 2):
        api.set_tuning("stream_k", v)
        sizes[v] = (ws(4096, 1024), ws(8192, 2048))
    assert sizes[2][0] > sizes[0][0] and sizes[2][1] == sizes[0][1]
    X = inputs.cov_inputs(4096, 1024, seed=37)["X"]
    got = host(api.correlation(dev(X), prec="3xbf16"))
    api.stream_check()
    assert inputs.rel_fro(got, oracle.correlation(X)) <= GATE
    A = inputs.int_matrix((1024, 4096), seed=38)
    C0 = inputs.int_matrix((1024, 1024), seed=39)
    ref = oracle.syrk(A, C0, 2.0, 1.0, 0)
    outs = []
    for v in (2, 0):
        api.set_tuning("stream_k", v)
        C = dev(C0)
        api.syrk(dev(A), C, 2.0, 1.0, prec="3xbf16")
        outs.append(host(C))
        api.stream_check()
    api.set_tuning("stream_k", 2)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], ref.astype(np.float32))


def test_streamk_graph_replay(api):
    """The stream-K flags are cleared inside the captured call: replays agree bit for bit."""
    api.set_tuning("stream_k", 1)
    g = inputs.gemm_inputs(1000, 1100, 1300, seed=36)
    A, B = dev(g["A"]), dev(g["B"])
    C = dev(g["C"])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        api.gemm(A, B, C, g["alpha"], 0.0, prec="3xbf16", stream=s)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        api.gemm(A, B, C, g["alpha"], 0.0, prec="3xbf16")
    outs = []
    for _ in range(3):
        C.fill_(float("nan"))
        graph.replay()
        outs.append(host(C))
    api.stream_check()
    api.set_tuning("stream_k", 2)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    ref = oracle.gemm(g["A"], g["B"], g["C"], g["alpha"], 0.0)
    assert inputs.rel_fro(outs[0], ref) <= GATE
