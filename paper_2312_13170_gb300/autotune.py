"""Autotuner for the engine knobs (tile width, accumulation chunk, CTA pairs,
staged beta input, stream-K; the FP32 tiled form's EXACT instance).

The runtime analogue of the compiler's tiling decision in loop
internalization (paper Sec. VI-C: the pass tiles the loop by the work-group
size): for a problem class -- operation, precision and a size bucket -- the
tuner times each candidate configuration through the C ABI on seeded
synthetic inputs of the call's shape, keeps the fastest, and caches it in a
JSON file keyed by GPU. The Python binding applies a cached choice before each
call (``LN_AUTOTUNE=cached``) and may search on a miss (``LN_AUTOTUNE=search``);
``LN_AUTOTUNE=off`` (the default) leaves the library's defaults in place.

Knobs (see ``ln_set_tuning`` in include/loopnest.h): ``tile_n`` in {0 (automatic), 128, 256}
for general contractions, ``chunk_kt`` in {1, 2} (k tiles accumulated in
tensor memory before promotion to FP32 registers), ``pair`` in {0, 1} (CTA
pairs with tcgen05.mma.cta_group::2), ``stage_beta`` in {0, 1}, ``stream_k``
in {0, 1, 2} (never, always, automatic), ``sym_wide`` in {0, 1, 2} (128 x 256
symmetric tiles: never, always, automatic), ``stage_out`` in {0, 1}, and for the FP32 tiled form ``simt_exact`` in {0, 1}
and ``simt_tile`` in {0 (automatic), 64, 128}. Batched
SYRK/SYR2K are tuned over ``chunk_kt`` (their 128 x 128 symmetric tiles and
stage count are fixed by the kernel's shared-memory plan). Only
configurations that keep the library's accuracy gate are offered; every one
gives a result within the gate, most bit-identical.

Cache: ``LN_AUTOTUNE_CACHE`` or ``~/.cache/libloopnest/autotune.json``.
"""
from __future__ import annotations

import json
import math
import os
import threading

import numpy as np

# tile_n 0 is the library's automatic width (256, or 128 for problems whose
# 256-wide tiles would fill at most half the SMs)
DEFAULT = {"tile_n": 0, "chunk_kt": 2, "pair": 1, "stage_beta": 1, "stream_k": 2, "simt_exact": 1, "sym_wide": 0, "stage_out": 1,
           "simt_tile": 0}


def _c(**kw):
    return dict(DEFAULT, **kw)


_GENERAL = [_c(), _c(tile_n=256), _c(tile_n=128), _c(chunk_kt=1), _c(pair=0), _c(stage_beta=0), _c(stream_k=1),
            _c(stream_k=0), _c(stage_out=0)]
_SYM = [_c(), _c(chunk_kt=1), _c(stream_k=1), _c(stream_k=0), _c(sym_wide=2), _c(sym_wide=1, stream_k=1)]
CANDIDATES = {
    "gemm": _GENERAL,
    "gemm_chain": _GENERAL,
    "three_mm": [_c(), _c(tile_n=128), _c(chunk_kt=1), _c(pair=0), _c(stream_k=1)],
    "covariance": _SYM,
    "correlation": _SYM,
    "syrk": _SYM,
    "syr2k": _SYM,
    "syrk_batched": [_c(), _c(chunk_kt=1)],
    "syr2k_batched": [_c(), _c(chunk_kt=1)],
}
# the FP32 tiled form (every operation): its EXACT instance or the general one,
# and either tile width
FP32_CANDIDATES = [_c(), _c(simt_exact=0), _c(simt_tile=64), _c(simt_tile=128)]


def candidates(op, prec):
    return FP32_CANDIDATES if prec == "fp32" else CANDIDATES[op]
_lock = threading.Lock()
_cache = None
_state = threading.local()  # set while a search runs, so its own calls are not re-tuned


def mode() -> str:
    m = os.environ.get("LN_AUTOTUNE", "off").lower()
    return m if m in ("off", "cached", "search") else "off"


def cache_path() -> str:
    return os.environ.get("LN_AUTOTUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "libloopnest", "autotune.json")


def bucket(shape) -> str:
    """Size bucket: each dimension rounded to the nearest power of two."""
    return "x".join(str(1 << max(0, int(round(math.log2(max(int(d), 1)))))) for d in shape)


def key(device: str, op: str, prec: str, shape) -> str:
    return f"{device}|{op}|{prec}|{bucket(shape)}"


def load(path=None) -> dict:
    global _cache
    path = path or cache_path()
    with _lock:
        if _cache is None or _cache.get("_path") != path:
            try:
                with open(path) as f:
                    _cache = json.load(f)
            except (OSError, ValueError):
                _cache = {}
            _cache["_path"] = path
        return _cache


def save(cache: dict, path=None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    data = {k: v for k, v in cache.items() if k != "_path"}
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def select(candidates, timer, reps=5, margin=0.03):
    """Time every candidate with timer(config) -> seconds (median of `reps`)
    and return (best_config, {index: median_seconds}). The first candidate
    (the library defaults) stays unless the fastest beats it by more than
    `margin`, so that call-to-call noise does not pick an equivalent
    configuration."""
    times = {}
    for i, cfg in enumerate(candidates):
        ts = sorted(timer(cfg) for _ in range(reps))
        times[i] = ts[len(ts) // 2]
    best = min(times, key=times.get)
    if times[best] > (1.0 - margin) * times[0]:
        best = 0
    return dict(candidates[best]), times


# ---------------------------------------------------------------- GPU side
def _device_name():
    import torch

    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}/{p.multi_processor_count}sm"


def _apply_config(cfg):
    from . import api

    for k in DEFAULT:
        api.set_tuning(k, int(cfg.get(k, DEFAULT[k])))


def _runner(op, shape, prec):
    """A callable that runs `op` once on synthetic inputs of `shape`."""
    import torch

    from . import api, inputs

    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(a).to(dev)
    if op == "gemm":
        M, N, K = shape
        d = inputs.gemm_inputs(M, N, K, seed=0)
        A, B, C = t(d["A"]), t(d["B"]), t(d["C"])
        return lambda: api.gemm(A, B, C, 1.0, 0.0, prec=prec)
    if op == "gemm_chain":
        ni, nj, nk, nl = shape
        d = inputs.chain_inputs(ni, nj, nk, nl, seed=0)
        A, B, C, D = (t(d[k]) for k in "ABCD")
        return lambda: api.gemm_chain(A, B, C, D, 1.5, 1.2, prec=prec)
    if op in ("covariance", "correlation"):
        n, m = shape
        X = t(inputs.cov_inputs(n, m, seed=0)["X"])
        fn = api.covariance if op == "covariance" else api.correlation
        return lambda: fn(X, prec=prec)
    if op in ("syrk", "syr2k"):
        n, k = shape
        d = inputs.sym_inputs(n, k, seed=0)
        A, B, C = t(d["A"]), t(d["B"]), t(d["C"])
        if op == "syrk":
            return lambda: api.syrk(A, C, 1.0, 0.0, prec=prec)
        return lambda: api.syr2k(A, B, C, 1.0, 0.0, prec=prec)
    if op == "three_mm":
        ni, nj, nk, nl, nm = shape
        rng = np.random.default_rng(0)
        A, B, C, D = (t(rng.uniform(-1, 1, size=s).astype(np.float32))
                      for s in ((ni, nk), (nk, nj), (nj, nm), (nm, nl)))
        return lambda: api.three_mm(A, B, C, D, prec=prec)
    if op in ("syrk_batched", "syr2k_batched"):
        # a batch of `count` instances of the class's mean sizes
        count, n, k = shape
        rng = np.random.default_rng(0)
        As = [t(rng.uniform(-1, 1, size=(n, k)).astype(np.float32)) for _ in range(count)]
        Bs = [t(rng.uniform(-1, 1, size=(n, k)).astype(np.float32)) for _ in range(count)] \
            if op == "syr2k_batched" else None
        Cs = [t(np.zeros((n, n), np.float32)) for _ in range(count)]
        batch = api.SymBatch(As, Cs, Bs, 1.0, 0.0, prec=prec)
        return batch.run
    raise ValueError(f"no tuner for {op}")


def tune(op, shape, prec="3xbf16", reps=5, save_result=True):
    """Search the candidates of `op` for `shape`; returns the chosen config."""
    import torch

    run = _runner(op, shape, prec)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timer(cfg):
        _apply_config(cfg)
        run()  # warm (also sizes the workspace for this configuration)
        start.record()
        run()
        stop.record()
        torch.cuda.synchronize()
        return start.elapsed_time(stop) / 1e3

    _state.active = True
    try:
        best, times = select(candidates(op, prec), timer, reps)
    finally:
        _state.active = False
        _apply_config(DEFAULT)
    if save_result:
        cache = load()
        cache[key(_device_name(), op, prec, shape)] = {"config": best, "seconds": times}
        save(cache)
    return best


def apply(op, shape, prec):
    """Apply the tuned configuration for this call (per LN_AUTOTUNE)."""
    m = mode()
    if m == "off" or getattr(_state, "active", False):
        return
    k = key(_device_name(), op, prec, shape)
    entry = load().get(k)
    if entry is None and m == "search" and op in CANDIDATES:
        tune(op, shape, prec)
        entry = load().get(k)
    _apply_config(entry["config"] if entry else DEFAULT)
