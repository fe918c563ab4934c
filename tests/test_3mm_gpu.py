"""GPU parity of the three chained products (polybench 3mm): G = (A B)(C D).

Forms and precisions as for the other contractions (gate 1e-5 relative
Frobenius against the FP64 oracle; single-pass BF16 loosely), sizes spanning
several tiles with ragged tails, integer inputs bit for bit, empty inner
dimensions, and pinned host operands.
"""
import numpy as np
import pytest

import oracle
from paper_2312_13170_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = 1e-5
MODES = [("plain", "fp32"), ("internalized", "fp32"), ("internalized", "bf16"), ("internalized", "3xbf16"),
         ("internalized", "6xbf16"), ("internalized", "tf32"), ("internalized", "3xtf32")]


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


def uni(shape, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=shape).astype(np.float32)


@pytest.mark.parametrize("form,prec", MODES)
@pytest.mark.parametrize("ni,nj,nk,nl,nm", [(1, 1, 1, 1, 1), (65, 127, 33, 129, 71), (200, 136, 264, 92, 150),
                                            (256, 256, 256, 256, 256)])
def test_3mm(api, form, prec, ni, nj, nk, nl, nm):
    A, B, C, D = uni((ni, nk), 1), uni((nk, nj), 2), uni((nj, nm), 3), uni((nm, nl), 4)
    ref = oracle.three_mm(A, B, C, D)
    G = api.three_mm(dev(A), dev(B), dev(C), dev(D), form=form, prec=prec)
    api.stream_check()
    assert inputs.rel_fro(host(G), ref) <= (3e-2 if prec in ("bf16", "tf32") else GATE)


@pytest.mark.parametrize("form,prec", [m for m in MODES if m[1] not in ("bf16", "tf32")])
def test_3mm_integer_bitexact(api, form, prec):
    # |E|, |F| <= 15 * 16 < 256 (one BF16 term, one TF32 term), |G| <= 200 * 240^2 < 2^24
    ni, nj, nk, nl, nm = 150, 200, 15, 130, 15
    A, B, C, D = (inputs.int_matrix(s, seed=90 + i) for i, s in enumerate([(ni, nk), (nk, nj), (nj, nm), (nm, nl)]))
    ref = oracle.three_mm(A, B, C, D)
    G = api.three_mm(dev(A), dev(B), dev(C), dev(D), form=form, prec=prec)
    api.stream_check()
    assert np.array_equal(host(G).astype(np.float64), ref)


def test_3mm_empty_inner_and_host_operands(api):
    A, B, C, D = uni((40, 0), 5), uni((0, 30), 6), uni((30, 20), 7), uni((20, 50), 8)
    G = dev(np.full((40, 50), np.nan, np.float32))
    api.three_mm(dev(A), dev(B), dev(C), dev(D), out=G)
    assert np.array_equal(host(G), np.zeros((40, 50), np.float32))
    A, B, C, D = uni((300, 200), 9), uni((200, 260), 10), uni((260, 180), 11), uni((180, 240), 12)
    Gd = api.three_mm(dev(A), dev(B), dev(C), dev(D), prec="3xbf16")
    hp = [torch.from_numpy(x).pin_memory() for x in (A, B, C, D)]
    Gh = api.three_mm(*hp, prec="3xbf16")
    api.stream_check()
    assert not Gh.is_cuda and torch.equal(Gh, Gd.cpu())
    assert inputs.rel_fro(Gh.numpy(), oracle.three_mm(A, B, C, D)) <= GATE


@pytest.mark.parametrize("form,prec", [("plain", "fp32"), ("internalized", "fp32"), ("internalized", "3xbf16"),
                                       ("internalized", "6xbf16"), ("internalized", "3xtf32")])
@pytest.mark.parametrize("ni,nj,nk,nl,nm", [(70, 129, 65, 90, 33), (1024, 1024, 1024, 1024, 1024)])
def test_3mm_bwd(api, form, prec, ni, nj, nk, nl, nm):
    if form == "plain" and ni > 512:
        pytest.skip("plain form at the large size is slow and adds nothing")
    A, B, C, D, Gb = uni((ni, nk), 21), uni((nk, nj), 22), uni((nj, nm), 23), uni((nm, nl), 24), uni((ni, nl), 25)
    ref = oracle.three_mm_vjp(A, B, C, D, Gb)
    got = api.three_mm_bwd(dev(A), dev(B), dev(C), dev(D), dev(Gb), form=form, prec=prec)
    api.stream_check()
    for g, r in zip(got, ref):
        assert inputs.rel_fro(host(g), r) <= GATE


def test_3mm_autograd(api):
    A, B, C, D = (dev(uni(s, 30 + i)).requires_grad_(True) for i, s in
                  enumerate([(96, 80), (80, 72), (72, 88), (88, 64)]))
    W = dev(uni((96, 64), 35))
    G = api.ThreeMmFn.apply(A, B, C, D, "internalized", "3xbf16")
    (G * W).sum().backward()
    ref = oracle.three_mm_vjp(*(host(t) for t in (A, B, C, D)), host(W))
    for t, r in zip((A, B, C, D), ref):
        assert inputs.rel_fro(host(t.grad), r) <= GATE
