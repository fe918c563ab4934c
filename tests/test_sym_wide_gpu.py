"""128 x 256 lower-triangle tiles of the symmetric contractions (the "sym_wide"
knob): covariance, correlation, SYRK and SYR2K with the wide tiles forced on
(1) agree with the FP64 oracle within the 1e-5 gate, bit for bit on integer
inputs against the 128 x 128 tiles (0), in every fill, at sizes with an odd
number of 128-row tiles (the packed operand is padded by one zero tile) and
ragged edges, with and without stream-K. The automatic setting (2) takes them
for the 8192 x 2048 covariance (72 wide tiles of 128 k-tiles: stream-K) and
not for a shallow SYRK; the default (0) never does."""
import ctypes

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
    a.set_tuning("sym_wide", 0)
    a.set_tuning("stream_k", 2)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def with_knobs(api, fn, **knobs):
    for k, v in knobs.items():
        api.set_tuning(k, v)
    try:
        out = fn()
        api.stream_check()
        return out
    finally:
        api.set_tuning("sym_wide", 0)
        api.set_tuning("stream_k", 2)


@pytest.mark.parametrize("prec", ["3xbf16", "bf16", "3xtf32"])
@pytest.mark.parametrize("fill", ["full", "lower", "upper"])
@pytest.mark.parametrize("sk", [0, 1])
def test_syrk_syr2k_wide_integer_bitexact(api, prec, fill, sk):
    n, k = 5 * 128 + 37, 300  # 6 row tiles: 3 row-tile pairs; ragged last tile
    A, B = inputs.int_matrix((n, k), seed=41), inputs.int_matrix((n, k), seed=42)
    C = inputs.int_matrix((n, n), seed=43)
    fl = {"full": 0, "lower": 1, "upper": 2}[fill]

    def run():
        C1, C2 = dev(C), dev(C)
        api.syrk(dev(A), C1, 2.0, -1.0, fill=fill, prec=prec)
        api.syr2k(dev(A), dev(B), C2, 2.0, -1.0, fill=fill, prec=prec)
        return host(C1), host(C2)

    w1, w2 = with_knobs(api, run, sym_wide=1, stream_k=sk)
    s1, s2 = with_knobs(api, run, sym_wide=0, stream_k=sk)
    assert np.array_equal(w1, s1) and np.array_equal(w2, s2)
    assert np.array_equal(w1.astype(np.float64), oracle.syrk(A, C, 2.0, -1.0, fl))
    assert np.array_equal(w2.astype(np.float64), oracle.syr2k(A, B, C, 2.0, -1.0, fl))


@pytest.mark.parametrize("n,m", [(3000, 700), (2500, 1100), (1000, 129)])
@pytest.mark.parametrize("prec", ["3xbf16", "3xtf32"])
def test_cov_corr_wide(api, n, m, prec):
    X = inputs.cov_inputs(n, m, seed=44)["X"]
    Xd = dev(X)
    cov_ref, corr_ref = oracle.covariance(X), oracle.correlation(X)
    for sk in (1, 0):
        c, r = with_knobs(api, lambda: (host(api.covariance(Xd, prec=prec)), host(api.correlation(Xd, prec=prec))),
                          sym_wide=1, stream_k=sk)
        assert inputs.rel_fro(c, cov_ref) <= GATE and inputs.rel_fro(r, corr_ref) <= GATE
        assert np.array_equal(c, c.T) and np.array_equal(r, r.T) and np.all(np.diag(r) == 1.0)


def test_sym_wide_default_policy(api):
    def ws(fn, *a):
        b = ctypes.c_size_t()
        assert fn(*a, ctypes.byref(b)) == 0
        return b.value

    L = api.lib()
    assert api.get_tuning("sym_wide") == 0
    sizes = {}
    for v in (0, 2):
        api.set_tuning("sym_wide", v)
        sizes[v] = (ws(L.ln_covariance_workspace_size, 8192, 2048, 1, 2), ws(L.ln_syrk_workspace_size, 2048, 64, 1, 2))
    api.set_tuning("sym_wide", 2)
    # the 8192 x 2048 covariance takes wide tiles (its stream-K partials are 256 wide)
    assert sizes[2][0] > sizes[0][0]
    # a shallow SYRK does not
    assert sizes[2][1] == sizes[0][1]
    X = inputs.cov_inputs(8192, 2048, seed=0)["X"]
    rows = np.array([0, 1, 500, 1023, 1500, 2047])
    got = host(api.covariance(dev(X), prec="3xbf16"))
    api.stream_check()
    api.set_tuning("sym_wide", 0)
    assert inputs.rel_fro(got[rows], oracle.cov_rows(X, rows)) <= GATE
