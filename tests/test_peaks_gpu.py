"""Peak probes (ln_peak_probe): each runs, reports no timeout, and measures a
rate inside the range the GB300's unit counts and clocks allow. The copy
probe must copy exactly.

Bounds: BF16 tcgen05 at most 152 SMs x 8192 flops per clock x 2.07 GHz
(2.58 PFLOP/s) and above 1 PFLOP/s; TF32 is half the BF16 rate per
instruction K (0.4-0.6 of the BF16 probe); FFMA at most 152 x 128 lanes x 2
flops x 2.07 GHz (80.5 TFLOP/s); HBM3e at most 8 TB/s.
"""
import pytest

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


def rate(api, kind, iters, src=None, dst=None, reps=5):
    """Median of event-timed launches: work per second."""
    api.peak_probe(kind, iters, src, dst)  # warm
    torch.cuda.synchronize()
    out = []
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        work = api.peak_probe(kind, iters, src, dst)
        e.record()
        e.synchronize()
        out.append(work / (s.elapsed_time(e) / 1e3))
    out.sort()
    return out[len(out) // 2]


def test_mma_probes(api):
    err = torch.ones(4, dtype=torch.int32, device="cuda")
    bf16 = rate(api, "mma_bf16", 4096, dst=err) / 1e12
    assert int(err[0]) == 0
    tf32 = rate(api, "mma_tf32", 4096, dst=err) / 1e12
    assert int(err[0]) == 0
    api.stream_check()
    assert 1000 < bf16 < 2600, bf16
    assert 0.4 < tf32 / bf16 < 0.6, (tf32, bf16)


def test_ffma_probe(api):
    sink = torch.zeros(1, device="cuda")
    ffma = rate(api, "ffma", 1024, dst=sink) / 1e12
    assert float(sink[0]) == 0.0
    assert 40 < ffma < 81, ffma


def test_copy_probe(api):
    n = 64 << 20  # 256 MiB each way: larger than L2
    src = torch.randn(n, device="cuda")
    dst = torch.zeros(n, device="cuda")
    gbs = rate(api, "copy", 0, src, dst) / 1e9
    assert torch.equal(src, dst)
    assert 2000 < gbs < 8000, gbs
    tail = torch.zeros(n - 4, device="cuda")  # a size that is not the whole buffer
    api.peak_probe("copy", 0, src, tail)
    assert torch.equal(src[: n - 4], tail)
    with pytest.raises(RuntimeError):
        api.peak_probe("copy", 0, src, src)  # overlapping ranges are refused
