"""Autotuner: selection, bucketing and cache (CPU), and one tuning pass (GPU)."""
import json

import numpy as np
import pytest

from paper_2312_13170_gb300 import autotune, inputs


def test_bucket_and_key():
    assert autotune.bucket((2048, 2048, 2048)) == "2048x2048x2048"
    assert autotune.bucket((2800, 100, 1)) == "2048x128x1"  # nearest power of two in log2
    assert autotune.bucket((3000, 0, 90)) == "4096x1x64"
    assert autotune.key("GB300/152sm", "gemm", "3xbf16", (2000, 2100, 8)) == "GB300/152sm|gemm|3xbf16|2048x2048x8"


def test_select_picks_fastest_median():
    cands = [{"tile_n": 256}, {"tile_n": 128}, {"tile_n": 64}]
    cost = {256: [3.0, 1.0, 3.0], 128: [2.0, 2.0, 2.0], 64: [9.0, 0.1, 9.0]}
    calls = {k: iter(v) for k, v in cost.items()}
    best, times = autotune.select(cands, lambda c: next(calls[c["tile_n"]]), reps=3)
    assert best == {"tile_n": 128}  # medians 3.0, 2.0, 9.0
    assert times == {0: 3.0, 1: 2.0, 2: 9.0}


def test_select_keeps_defaults_within_margin():
    cands = [{"tile_n": 0}, {"tile_n": 128}, {"tile_n": 256}]
    cost = {0: 1.0, 128: 0.98, 256: 1.5}  # 2 % faster: within the 3 % margin
    best, _ = autotune.select(cands, lambda c: cost[c["tile_n"]], reps=1)
    assert best == {"tile_n": 0}
    cost[128] = 0.96
    best, _ = autotune.select(cands, lambda c: cost[c["tile_n"]], reps=1)
    assert best == {"tile_n": 128}
    best, _ = autotune.select(cands, lambda c: cost[c["tile_n"]], reps=1, margin=0.05)
    assert best == {"tile_n": 0}


def test_cache_roundtrip(tmp_path, monkeypatch):
    path = str(tmp_path / "tune.json")
    monkeypatch.setenv("LN_AUTOTUNE_CACHE", path)
    c = autotune.load()
    c["dev|gemm|3xbf16|256x256x256"] = {"config": {"tile_n": 128, "chunk_kt": 2}}
    autotune.save(c)
    data = json.load(open(path))
    assert data == {"dev|gemm|3xbf16|256x256x256": {"config": {"tile_n": 128, "chunk_kt": 2}}}
    monkeypatch.setenv("LN_AUTOTUNE", "bogus")
    assert autotune.mode() == "off"
    monkeypatch.setenv("LN_AUTOTUNE", "search")
    assert autotune.mode() == "search"


def test_candidates_respect_knob_domains():
    domains = {"tile_n": (0, 128, 256), "chunk_kt": (1, 2), "pair": (0, 1, 2), "stage_beta": (0, 1),
               "stream_k": (0, 1, 2), "simt_exact": (0, 1), "sym_wide": (0, 1, 2), "stage_out": (0, 1),
               "simt_tile": (0, 64, 128)}
    for op, cands in list(autotune.CANDIDATES.items()) + [("fp32", autotune.FP32_CANDIDATES)]:
        assert cands[0] == autotune.DEFAULT, op  # the library defaults are always a candidate
        for c in cands:
            assert set(c) == set(domains), (op, c)
            for k, v in c.items():
                assert v in domains[k], (op, c)
    assert autotune.candidates("gemm", "fp32") is autotune.FP32_CANDIDATES
    assert autotune.candidates("syrk_batched", "3xbf16") is autotune.CANDIDATES["syrk_batched"]


@pytest.mark.gpu
def test_tuning_pass_and_cached_use(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    import oracle

    __graft_entry__.build()
    from paper_2312_13170_gb300 import api

    monkeypatch.setenv("LN_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    shape = (300, 260, 200, 280)
    best = autotune.tune("gemm_chain", shape, "3xbf16", reps=3)
    assert best in autotune.CANDIDATES["gemm_chain"]
    assert all(api.get_tuning(k) == v for k, v in autotune.DEFAULT.items())  # defaults restored
    monkeypatch.setenv("LN_AUTOTUNE", "cached")
    d = inputs.chain_inputs(*shape, seed=3)
    t = {k: torch.from_numpy(d[k]).cuda() for k in "ABCD"}
    E, F = api.gemm_chain(t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], prec="3xbf16")
    assert api.get_tuning("tile_n") == best["tile_n"]
    E_ref, F_ref = oracle.gemm_chain(d["A"], d["B"], d["C"], d["D"], d["alpha"], d["beta"])
    assert inputs.rel_fro(F.cpu().numpy(), F_ref) <= 1e-5
    # every knob setting keeps the gate
    for cfg in autotune.CANDIDATES["gemm_chain"]:
        for k, v in cfg.items():
            api.set_tuning(k, v)
        E, F = api.gemm_chain(t["A"], t["B"], t["C"], t["D"], d["alpha"], d["beta"], prec="3xbf16")
        torch.cuda.synchronize()
        assert inputs.rel_fro(F.cpu().numpy(), F_ref) <= 1e-5, cfg
    for k, v in autotune.DEFAULT.items():
        api.set_tuning(k, v)


@pytest.mark.gpu
@pytest.mark.parametrize("tile_n,chunk_kt", [(128, 2), (256, 1), (128, 1)])
def test_knob_settings_keep_parity(tile_n, chunk_kt):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    import oracle

    __graft_entry__.build()
    from paper_2312_13170_gb300 import api

    api.set_tuning("tile_n", tile_n)
    api.set_tuning("chunk_kt", chunk_kt)
    try:
        g = inputs.gemm_inputs(333, 517, 389, seed=11)
        C = torch.from_numpy(g["C"]).cuda()
        api.gemm(torch.from_numpy(g["A"]).cuda(), torch.from_numpy(g["B"]).cuda(), C, g["alpha"], g["beta"],
                 prec="3xbf16")
        ref = oracle.gemm(g["A"], g["B"], g["C"], g["alpha"], g["beta"])
        assert inputs.rel_fro(C.cpu().numpy(), ref) <= 1e-5
        s = inputs.sym_inputs(301, 457, seed=12)
        C = torch.from_numpy(s["C"]).cuda()
        api.syrk(torch.from_numpy(s["A"]).cuda(), C, s["alpha"], s["beta"], prec="3xbf16")
        ref = oracle.syrk(s["A"], s["C"], s["alpha"], s["beta"])
        assert inputs.rel_fro(C.cpu().numpy(), ref) <= 1e-5
        X = inputs.cov_inputs(700, 300, seed=13)["X"]
        cov = api.covariance(torch.from_numpy(X).cuda(), prec="6xbf16")
        assert inputs.rel_fro(cov.cpu().numpy(), oracle.covariance(X)) <= 1e-5
    finally:
        api.set_tuning("tile_n", 0)
        api.set_tuning("chunk_kt", 2)


@pytest.mark.gpu
def test_tuning_batched_and_fp32(tmp_path, monkeypatch):
    """The batched path and the FP32 tiled form are tuned and cached too; the
    chosen configuration is applied before the call and keeps the gate."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    import oracle

    __graft_entry__.build()
    from paper_2312_13170_gb300 import api

    monkeypatch.setenv("LN_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    best = autotune.tune("syrk_batched", (6, 200, 90), "3xbf16", reps=2)
    assert best in autotune.CANDIDATES["syrk_batched"]
    best = autotune.tune("gemm", (256, 256, 256), "fp32", reps=2)
    assert best in autotune.FP32_CANDIDATES
    monkeypatch.setenv("LN_AUTOTUNE", "cached")
    g = inputs.gemm_inputs(256, 256, 256, seed=4)
    C = torch.from_numpy(g["C"]).cuda()
    api.gemm(torch.from_numpy(g["A"]).cuda(), torch.from_numpy(g["B"]).cuda(), C, g["alpha"], g["beta"],
             form="internalized", prec="fp32")
    assert api.get_tuning("simt_exact") == best["simt_exact"]
    assert inputs.rel_fro(C.cpu().numpy(), oracle.gemm(g["A"], g["B"], g["C"], g["alpha"], g["beta"])) <= 1e-5
    for k, v in autotune.DEFAULT.items():
        api.set_tuning(k, v)
