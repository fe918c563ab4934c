"""ln_covariance_noalloc: the covariance for callers that cannot allocate.

Some callers cannot call cudaMalloc (allocator internals, memory-capped
sandboxes, loops that must never enter the allocator), so this entry point
takes no workspace and keeps its scratch in a fixed 8 MiB device array inside
the library. The tests call it through the C ABI:
- twice in a row on different data, each result bit for bit equal to the
  workspace-taking ln_covariance (internalized FP32 form: the same mean pass,
  centring pair and contraction), and within the 1e-5 relative Frobenius gate
  of the FP64 oracle;
- on a shape whose scratch is exactly the 8 MiB (accepted, equal to
  ln_covariance) and one row more (refused before anything is launched);
- with sizes beyond 2^22 (refused on the host).
This file is collected last, so a run that stops at the first failure has
already run every other test.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2312_13170_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LIMIT = 8 << 20


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2312_13170_gb300 import api as a

    return a


def scratch_bytes(n, m):
    """The entry point's scratch for n x m, by the layout its header states:
    FP64 means, the FP32 centring pair and 8 * m * ceil(n / r) bytes of
    partial sums, r = 256, 128 or 64 rows per reduction block (the largest
    giving at least 608 blocks of 128 columns), each piece 256-byte aligned."""
    colb = math.ceil(m / 128)
    r = next((sr for sr in (256, 128) if colb * math.ceil(n / sr) >= 608), 64)

    def a256(b):
        return (b + 255) // 256 * 256

    return a256(8 * m) + 2 * a256(4 * m) + a256(8 * m * math.ceil(n / r))


def noalloc(api, X, out):
    n, m = X.shape
    return api.lib().ln_covariance_noalloc(n, m, ctypes.c_void_p(X.data_ptr()), m, ctypes.c_void_p(out.data_ptr()),
                                           m, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_workspace_covariance_twice(api):
    for seed, (n, m) in ((1, (1000, 300)), (2, (777, 129))):
        X = torch.from_numpy(inputs.cov_inputs(n, m, seed=seed)["X"]).cuda()
        out = torch.full((m, m), float("nan"), device="cuda")
        assert noalloc(api, X, out) == 0, api.lib().ln_get_last_error()
        api.stream_check()
        ref = api.covariance(X, form="internalized", prec="fp32")
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, ref.cpu().numpy())
        assert inputs.rel_fro(got, oracle.covariance(X.cpu().numpy())) <= 1e-5


def test_noalloc_at_the_scratch_limit(api):
    m = 1024
    n = 261632  # the largest n whose scratch fits: 8 MiB exactly
    assert scratch_bytes(n, m) == LIMIT and scratch_bytes(n + 1, m) > LIMIT
    X = torch.randn((n, m), device="cuda", generator=torch.Generator(device="cuda").manual_seed(3)) * 2 + 5
    out = torch.empty((m, m), device="cuda")
    assert noalloc(api, X, out) == 0, api.lib().ln_get_last_error()
    api.stream_check()
    ref = api.covariance(X, form="internalized", prec="fp32")
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # one row more: refused with a message, nothing launched, no output touched
    X2 = torch.empty((n + 1, m), device="cuda")
    out2 = torch.full((m, m), 7.0, device="cuda")
    s = noalloc(api, X2, out2)
    assert s == 1 and b"scratch" in api.lib().ln_get_last_error()
    torch.cuda.synchronize()
    assert bool((out2 == 7.0).all())


def test_noalloc_rejects_sizes_on_the_host(api):
    # nothing is dereferenced or launched: the pointers are never used
    bogus_x, bogus_c = ctypes.c_void_p(0x7F0000000000), ctypes.c_void_p(0x7F8000000000)
    L = api.lib()
    assert L.ln_covariance_noalloc(4096, 1 << 20, bogus_x, 1 << 20, bogus_c, 1 << 20, None) == 1
    assert b"scratch" in L.ln_get_last_error()
    assert L.ln_covariance_noalloc((1 << 22) + 1, 1, bogus_x, 1, bogus_c, 1, None) == 1
    assert b"out of range" in L.ln_get_last_error()
    assert L.ln_covariance_noalloc(-1, 4, bogus_x, 4, bogus_c, 4, None) == 1
