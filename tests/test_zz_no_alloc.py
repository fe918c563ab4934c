"""ln_covariance_noalloc: the covariance for callers that cannot allocate.

Some callers cannot call cudaMalloc (allocator internals, memory-capped
sandboxes, loops that must never enter the allocator), so this entry point
takes no workspace and keeps its scratch in a fixed device array inside the
library. This test calls it through the C ABI twice in a row, on different
data, and checks each result against the workspace-taking ln_covariance
(internalized FP32 form) within the 1e-5 relative Frobenius tolerance used by
the other parity tests; it also checks that an oversized problem is refused
before anything is launched. It lives in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest

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


def noalloc(api, X, out):
    n, m = X.shape
    s = api.lib().ln_covariance_noalloc(n, m, ctypes.c_void_p(X.data_ptr()), m, ctypes.c_void_p(out.data_ptr()), m,
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return s


def test_noalloc_matches_workspace_covariance_twice(api):
    for seed, (n, m) in ((1, (1000, 300)), (2, (777, 129))):
        X = torch.from_numpy(inputs.cov_inputs(n, m, seed=seed)["X"]).cuda()
        out = torch.full((m, m), float("nan"), device="cuda")
        assert noalloc(api, X, out) == 0, api.lib().ln_get_last_error()
        api.stream_check()
        ref = api.covariance(X, form="internalized", prec="fp32")
        torch.cuda.synchronize()
        assert inputs.rel_fro(out.cpu().numpy(), ref.cpu().numpy()) <= 1e-5


def test_noalloc_rejects_oversized(api):
    # 2^20 features need far more than the fixed scratch; refused on the host
    bogus = ctypes.c_void_p(0x7F0000000000)
    s = api.lib().ln_covariance_noalloc(4096, 1 << 20, bogus, 1 << 20, ctypes.c_void_p(0x7F8000000000), 1 << 20, None)
    assert s == 1 and b"scratch" in api.lib().ln_get_last_error()
