"""The internalized FP32 form (exact FFMA, cp.async-staged k-tiles in a
four-stage shared-memory ring; 64- or 128-wide tiles; an EXACT instance
specialised on whole tiles and aligned rows, the "simt_exact" knob; the tile
width is forced with the "simt_tile" knob).

Every layout the library uses (GEMM A[i][k] B[k][j]; covariance A[k][i]
B[k][j] with centring; SYRK A[i][k] B[j][k]; chain and 3mm intermediates) is
checked against the FP64 oracle at the 1e-5 gate, on shapes that take the
EXACT instance and on ragged, unaligned ones that do not; integer inputs must
be bit-exact, and the EXACT instance must equal the general one bit for bit.
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
    a.set_tuning("simt_exact", 1)
    a.set_tuning("simt_tile", 0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def both(api, fn):
    out = []
    for on in (1, 0):
        api.set_tuning("simt_exact", on)
        out.append(fn())
    api.set_tuning("simt_exact", 1)
    api.stream_check()
    return out


@pytest.mark.parametrize("M,N,K", [(256, 256, 256), (512, 384, 640), (1024, 1024, 1024), (300, 517, 389),
                                   (129, 1, 9), (64, 64, 8), (2048, 2048, 40)])
def test_gemm_fp32(api, M, N, K):
    g = inputs.gemm_inputs(M, N, K, seed=M * 7 + K)

    def run():
        C = dev(g["C"])
        api.gemm(dev(g["A"]), dev(g["B"]), C, g["alpha"], g["beta"], form="internalized", prec="fp32")
        return host(C)

    on, off = both(api, run)
    assert np.array_equal(on, off)
    assert inputs.rel_fro(on, oracle.gemm(g["A"], g["B"], g["C"], g["alpha"], g["beta"])) <= GATE


def test_gemm_fp32_unaligned_view(api):
    g = inputs.gemm_inputs(256, 256, 256, seed=3)
    big = torch.zeros((256, 257), device="cuda")
    big[:, 1:] = dev(g["A"])
    A = big[:, 1:]  # rows 4 bytes off 16-byte alignment: the general instance
    C = dev(g["C"])
    api.gemm(A, dev(g["B"]), C, g["alpha"], g["beta"], form="internalized", prec="fp32")
    assert inputs.rel_fro(host(C), oracle.gemm(g["A"], g["B"], g["C"], g["alpha"], g["beta"])) <= GATE


def test_gemm_fp32_integer_bitexact(api):
    A, B, C = inputs.int_matrix((384, 512), seed=1), inputs.int_matrix((512, 256), seed=2), inputs.int_matrix(
        (384, 256), seed=3)
    Cd = dev(C)
    api.gemm(dev(A), dev(B), Cd, 2.0, -1.0, form="internalized", prec="fp32")
    assert np.array_equal(host(Cd).astype(np.float64), oracle.gemm(A, B, C, 2.0, -1.0))


@pytest.mark.parametrize("n,m", [(1024, 256), (1000, 300), (8192, 128)])
def test_cov_corr_fp32(api, n, m):
    X = inputs.cov_inputs(n, m, seed=n + m)["X"]
    Xd = dev(X)
    (c1, r1), (c0, r0) = both(api, lambda: (host(api.covariance(Xd, form="internalized", prec="fp32")),
                                             host(api.correlation(Xd, form="internalized", prec="fp32"))))
    assert np.array_equal(c1, c0) and np.array_equal(r1, r0)
    assert inputs.rel_fro(c1, oracle.covariance(X)) <= GATE
    assert inputs.rel_fro(r1, oracle.correlation(X)) <= GATE


@pytest.mark.parametrize("fill", ["full", "lower", "upper"])
@pytest.mark.parametrize("n,k", [(256, 128), (300, 77), (1024, 512)])
def test_syrk_syr2k_fp32(api, fill, n, k):
    d = inputs.sym_inputs(n, k, seed=n + 3 * k)
    fl = {"full": 0, "lower": 1, "upper": 2}[fill]

    def run():
        C1, C2 = dev(d["C"]), dev(d["C"])
        api.syrk(dev(d["A"]), C1, d["alpha"], d["beta"], fill=fill, form="internalized", prec="fp32")
        api.syr2k(dev(d["A"]), dev(d["B"]), C2, d["alpha"], d["beta"], fill=fill, form="internalized", prec="fp32")
        return host(C1), host(C2)

    (a1, a2), (b1, b2) = both(api, run)
    assert np.array_equal(a1, b1) and np.array_equal(a2, b2)
    assert inputs.rel_fro(a1, oracle.syrk(d["A"], d["C"], d["alpha"], d["beta"], fl)) <= GATE
    assert inputs.rel_fro(a2, oracle.syr2k(d["A"], d["B"], d["C"], d["alpha"], d["beta"], fl)) <= GATE


def test_chain_fp32(api):
    d = inputs.chain_inputs(512, 384, 256, 640, seed=9)
    t = {k: dev(d[k]) for k in "ABCD"}
    (E1, F1), (E0, F0) = both(api, lambda: tuple(host(x) for x in api.gemm_chain(
        t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], form="internalized", prec="fp32")))
    assert np.array_equal(E1, E0) and np.array_equal(F1, F0)
    E_ref, F_ref = oracle.gemm_chain(d["A"], d["B"], d["C"], d["D"], d["alpha"], d["beta"])
    assert inputs.rel_fro(E1, E_ref) <= GATE and inputs.rel_fro(F1, F_ref) <= GATE


@pytest.mark.parametrize("M,N,K", [(1024, 1024, 512), (300, 517, 389), (2048, 2048, 64)])
def test_tile_width_bit_identical(api, M, N, K):
    """Each output is one FFMA chain over k in order, whatever the CTA tile:
    64- and 128-wide tiles give the same bits, GEMM and symmetric outputs."""
    g = inputs.gemm_inputs(M, N, K, seed=M + K)
    d = inputs.sym_inputs(M, K, seed=N)
    out = []
    try:
        for tb in (64, 128):
            api.set_tuning("simt_tile", tb)
            C = dev(g["C"])
            api.gemm(dev(g["A"]), dev(g["B"]), C, g["alpha"], g["beta"], form="internalized", prec="fp32")
            S = dev(d["C"])
            api.syrk(dev(d["A"]), S, d["alpha"], d["beta"], fill="lower", form="internalized", prec="fp32")
            api.stream_check()
            out.append((host(C), host(S)))
    finally:
        api.set_tuning("simt_tile", 0)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert inputs.rel_fro(out[0][0], oracle.gemm(g["A"], g["B"], g["C"], g["alpha"], g["beta"])) <= GATE
    assert inputs.rel_fro(out[0][1], oracle.syrk(d["A"], d["C"], d["alpha"], d["beta"], 1)) <= GATE
