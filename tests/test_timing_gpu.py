"""Launch timing through the C ABI (ln_timing_enable / ln_timing_read).

Mode 1 brackets every launch with its own event pair; mode 2 lets the chain's
two tensor-core contractions, which the library launches back to back on one
stream with programmatic overlap, share one pair. Both count every launch, both
work eagerly and inside a captured graph (the events become graph nodes), and
neither changes the result. The span of the two contractions cannot be shorter
than the second one alone, nor (beyond timer noise) longer than the two
bracketed launches together.
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

    yield a
    a.timing_enable(0)


FAMS = ("umma", "pack", "simt", "plain", "stats")


def clear(api):
    for f in FAMS:
        api.timing_read(f)


def test_modes_count_launches_and_keep_results(api):
    d = inputs.chain_inputs(2048, 2048, 2048, 2048, seed=51)
    t = {k: torch.from_numpy(d[k]).cuda() for k in "ABCD"}
    out, got = {}, {}
    for mode in (0, 1, 2):
        api.timing_enable(mode)
        clear(api)
        l0 = api.launch_count()
        E, F = api.gemm_chain(t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], prec="3xbf16")
        launches = api.launch_count() - l0
        torch.cuda.synchronize()
        got[mode] = {f: api.timing_read(f) for f in ("umma", "pack")}
        out[mode] = (E.cpu().numpy(), F.cpu().numpy())
        api.timing_enable(0)
        assert got[mode]["umma"][1] == (2 if mode else 0)
        if mode:
            assert got[mode]["umma"][1] + got[mode]["pack"][1] <= launches
    api.stream_check()
    for mode in (1, 2):
        assert np.array_equal(out[mode][0], out[0][0]) and np.array_equal(out[mode][1], out[0][1])
    assert got[1]["umma"][0] > 0 and got[2]["umma"][0] > 0
    rows = slice(0, 16)
    E_ref, _ = oracle.gemm_chain(d["A"][rows], d["B"], d["C"], d["D"][rows], d["alpha"], d["beta"])
    assert inputs.rel_fro(out[2][0][rows], E_ref) <= 1e-5


def test_span_in_graph_replay(api):
    d = inputs.chain_inputs(2048, 2048, 2048, 2048, seed=52)
    t = {k: torch.from_numpy(d[k]).cuda() for k in "ABCD"}
    E = torch.empty((2048, 2048), device="cuda")
    F = torch.empty_like(E)

    def call():
        api.gemm_chain(t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], prec="3xbf16", out=(E, F))

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        call()  # warm: workspace and shared-memory opt-ins before capture
    torch.cuda.current_stream().wait_stream(s)
    res = {}
    for mode in (1, 2):
        api.timing_enable(mode)
        clear(api)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            call()
        api.timing_enable(0)
        for _ in range(3):  # the event nodes keep the latest replay's times
            g.replay()
        torch.cuda.synchronize()
        ms, n = api.timing_read("umma")  # read once: the events go back to the library's pool
        assert n == 2 and ms > 0, (mode, ms, n)
        res[mode] = ms
        del g
    api.stream_check()
    # the span holds both contractions: more than one alone, and not more
    # than the two launches with an event pair each (20 % slack for noise)
    assert res[2] > 0.5 * res[1] and res[2] <= 1.2 * res[1], res
    E_ref, _ = oracle.gemm_chain(d["A"][:8], d["B"], d["C"], d["D"][:8], d["alpha"], d["beta"])
    assert inputs.rel_fro(E[:8].cpu().numpy(), E_ref) <= 1e-5
