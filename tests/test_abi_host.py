"""Host-side checks of the C ABI (no GPU needed).

The library must load and export every entry point declared in
include/loopnest.h, and argument validation, aliasing checks and workspace
queries must behave as the header states. The pointers used here are fake
device addresses that the library never dereferences: every call below fails
validation (or is a size query) before any CUDA call is made.
"""
import ctypes
import os
import re

import pytest

from paper_2312_13170_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "loopnest.h")


@pytest.fixture(scope="module")
def L():
    build.build()
    return api.lib()


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ln_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported(L):
    names = declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(L, n), f"{n} declared in loopnest.h but not exported"
    assert set(names) == set(api.EXPORTS), "binding and header disagree"


def test_version_and_status_strings(L):
    assert L.ln_version() >= 100
    assert L.ln_status_string(2) == b"LN_ERR_ALIASING"
    assert L.ln_status_string(99) == b"LN_UNKNOWN_STATUS"


FAKE_A = 0x7F0000000000
FAKE_B = 0x7F0000100000
FAKE_C = 0x7F0000200000


def P(x):
    return ctypes.c_void_p(x)


def last(L):
    return L.ln_get_last_error().decode()


def test_gemm_validation(L):
    # negative size
    assert L.ln_gemm(-1, 4, 4, 1.0, P(FAKE_A), 4, P(FAKE_B), 4, 0.0, P(FAKE_C), 4, None, 0, 0, 0, None) == 1
    # ld smaller than the column count
    assert L.ln_gemm(4, 4, 4, 1.0, P(FAKE_A), 3, P(FAKE_B), 4, 0.0, P(FAKE_C), 4, None, 0, 0, 0, None) == 1
    # NULL operand
    assert L.ln_gemm(4, 4, 4, 1.0, None, 4, P(FAKE_B), 4, 0.0, P(FAKE_C), 4, None, 0, 0, 0, None) == 1
    # C overlapping A -> aliasing (the alias contract of the transformation)
    s = L.ln_gemm(64, 64, 64, 1.0, P(FAKE_A), 64, P(FAKE_B), 64, 0.0, P(FAKE_A + 256), 64, None, 0, 0, 0, None)
    assert s == 2 and "overlap" in last(L)
    # plain form supports only FP32 (the TF32 modes too are tensor-core only)
    assert L.ln_gemm(4, 4, 4, 1.0, P(FAKE_A), 4, P(FAKE_B), 4, 0.0, P(FAKE_C), 4, None, 0, 0, 2, None) == 4
    assert L.ln_gemm(4, 4, 4, 1.0, P(FAKE_A), 4, P(FAKE_B), 4, 0.0, P(FAKE_C), 4, None, 0, 0, 5, None) == 4
    # precision codes end at LN_PREC_3XTF32 = 5
    assert L.ln_gemm(4, 4, 4, 1.0, P(FAKE_A), 4, P(FAKE_B), 4, 0.0, P(FAKE_C), 4, None, 0, 1, 6, None) == 1
    # unknown enum
    assert L.ln_gemm(4, 4, 4, 1.0, P(FAKE_A), 4, P(FAKE_B), 4, 0.0, P(FAKE_C), 4, None, 0, 7, 0, None) == 1
    # tensor-core path without a workspace
    s = L.ln_gemm(256, 256, 256, 1.0, P(FAKE_A), 256, P(FAKE_B), 256, 0.0, P(FAKE_C), 256, None, 0, 1, 2, None)
    assert s == 7 and "workspace" in last(L)
    # zero-size is a no-op that succeeds without touching anything
    assert L.ln_gemm(0, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, None, 0, 1, 2, None) == 0


def test_workspace_queries(L):
    # the automatic tile width depends on the GPU's SM count: pin 256-wide tiles
    old = ctypes.c_int(0)
    assert L.ln_get_tuning(b"tile_n", ctypes.byref(old)) == 0
    assert L.ln_set_tuning(b"tile_n", 256) == 0
    try:
        _workspace_queries_256(L)
    finally:
        L.ln_set_tuning(b"tile_n", old.value)


def _workspace_queries_256(L):
    n = ctypes.c_size_t()
    assert L.ln_gemm_workspace_size(256, 256, 256, 0, 0, ctypes.byref(n)) == 0 and n.value == 0
    assert L.ln_gemm_workspace_size(256, 256, 256, 1, 0, ctypes.byref(n)) == 0 and n.value == 0
    assert L.ln_gemm_workspace_size(256, 256, 256, 1, 2, ctypes.byref(n)) == 0
    # two packed operands of 2 row tiles x 4 k-tiles x 2 terms x 16 KiB
    assert n.value == 2 * (2 * 4 * 2 * 16384)
    # N = 100 -> one 256-wide column tile, so the N side is padded to 2 row tiles
    assert L.ln_gemm_workspace_size(200, 100, 70, 1, 2, ctypes.byref(n)) == 0
    assert n.value == (2 * 2 * 2 + 2 * 2 * 2) * 16384
    # three split terms use 128-wide tiles: no padding
    assert L.ln_gemm_workspace_size(200, 100, 70, 1, 3, ctypes.byref(n)) == 0
    assert n.value == (2 * 2 * 3 + 1 * 2 * 3) * 16384
    assert L.ln_gemm_chain_workspace_size(2048, 2048, 2048, 2048, 1, 2, ctypes.byref(n)) == 0
    # packed A, B^T, T (written by the first contraction's epilogue) and C^T; no FP32 T
    assert n.value == 4 * (16 * 32 * 2 * 16384)
    assert L.ln_gemm_chain_workspace_size(2048, 2048, 2048, 2048, 1, 0, ctypes.byref(n)) == 0
    assert n.value == 4 * 2048 * 2048
    assert L.ln_covariance_workspace_size(8192, 2048, 1, 2, ctypes.byref(n)) == 0 and n.value > 0
    assert L.ln_syr2k_workspace_size(100, 50, 1, 2, ctypes.byref(n)) == 0 and n.value == 2 * 2 * 16384
    # TF32 terms take 4 bytes: one TF32 term packs into as many bytes as two BF16 terms
    assert L.ln_syr2k_workspace_size(100, 50, 1, 4, ctypes.byref(n)) == 0 and n.value == 2 * 2 * 16384
    assert L.ln_syr2k_workspace_size(100, 50, 1, 5, ctypes.byref(n)) == 0 and n.value == 2 * 4 * 16384


def test_sym_validation(L):
    s = L.ln_syrk(5, 8, 8, 1.0, P(FAKE_A), 8, 0.0, P(FAKE_C), 8, None, 0, 0, 0, None)
    assert s == 1 and "fill" in last(L)
    s = L.ln_syr2k(0, 64, 64, 1.0, P(FAKE_A), 64, P(FAKE_B), 64, 0.0, P(FAKE_B + 1024), 64, None, 0, 0, 0, None)
    assert s == 2


def test_cov_validation(L):
    assert L.ln_covariance(1, 8, P(FAKE_A), 8, P(FAKE_C), 8, None, 0, 0, 0, None) == 1
    assert L.ln_correlation(16, 8, P(FAKE_A), 8, P(FAKE_A + 64), 8, None, 0, 0, 0, None) == 2
    # the statistics-returning forms: NULL, overlapping X or the output, misaligned
    assert L.ln_covariance_fwd(16, 8, P(FAKE_A), 8, P(FAKE_C), 8, None, None, 0, 1, 2, None) == 1
    assert "statistics" in last(L)
    assert L.ln_correlation_fwd(16, 8, P(FAKE_A), 8, P(FAKE_C), 8, P(FAKE_A + 8), None, 0, 1, 2, None) == 2
    assert L.ln_correlation_fwd(16, 8, P(FAKE_A), 8, P(FAKE_C), 8, P(FAKE_C + 64), None, 0, 1, 2, None) == 2
    assert L.ln_covariance_fwd(16, 8, P(FAKE_A), 8, P(FAKE_C), 8, P(FAKE_B + 4), None, 0, 1, 2, None) == 1
    # a valid call without a workspace stops at the workspace check, before any launch
    assert L.ln_covariance_fwd(16, 8, P(FAKE_A), 8, P(FAKE_C), 8, P(FAKE_B), None, 0, 1, 2, None) == 7


def test_batched_validation(L):
    descs = (api.SymDesc * 2)()
    descs[0] = api.SymDesc(64, 32, FAKE_A, 32, None, 0, FAKE_C, 64)
    descs[1] = api.SymDesc(64, 32, FAKE_B, 32, None, 0, FAKE_C + 1024, 64)  # overlaps instance 0's C
    n = ctypes.c_size_t()
    assert L.ln_syrk_batched_workspace_size(2, ctypes.byref(descs), 1, 2, ctypes.byref(n)) == 2
    descs[1] = api.SymDesc(64, 32, FAKE_B, 32, None, 0, FAKE_C + 64 * 64 * 4, 64)
    assert L.ln_syrk_batched_workspace_size(2, ctypes.byref(descs), 1, 2, ctypes.byref(n)) == 0
    # rank-ordered packed operands: 2 instances x 1 row tile x 1 k tile x 2 terms, plus descriptors
    assert n.value >= 2 * 2 * 16384
    descs[1] = api.SymDesc(64, 32, FAKE_C + 4, 32, None, 0, FAKE_C + 64 * 64 * 4, 64)  # input inside an output
    assert L.ln_syrk_batched_workspace_size(2, ctypes.byref(descs), 1, 2, ctypes.byref(n)) == 2


def test_stream_check_symbol_present(L):
    assert callable(L.ln_stream_check)


def test_3mm_validation_and_workspace(L):
    FAKE_D, FAKE_G = 0x7F0000300000, 0x7F0000400000
    ws = ctypes.c_size_t(0)
    # negative size, bad form, NULL operand, G aliasing an input
    assert L.ln_3mm(-1, 4, 4, 4, 4, P(FAKE_A), P(FAKE_B), P(FAKE_C), P(FAKE_D), P(FAKE_G), None, 0, 1, 2, None) == 1
    assert L.ln_3mm(4, 4, 4, 4, 4, P(FAKE_A), P(FAKE_B), P(FAKE_C), P(FAKE_D), P(FAKE_G), None, 0, 7, 2, None) == 1
    assert L.ln_3mm(4, 4, 4, 4, 4, P(FAKE_A), None, P(FAKE_C), P(FAKE_D), P(FAKE_G), None, 0, 1, 2, None) == 1
    assert "NULL" in last(L)
    assert L.ln_3mm(8, 8, 8, 8, 8, P(FAKE_A), P(FAKE_B), P(FAKE_C), P(FAKE_D), P(FAKE_A + 64), None, 0, 1, 2,
                    None) == 2
    # empty outputs are a no-op
    assert L.ln_3mm(0, 4, 4, 4, 4, None, None, None, None, None, None, 0, 1, 2, None) == 0
    # FP32 forms keep E (ni x nj) and F (nj x nl) in the workspace, 256-byte aligned each
    assert L.ln_3mm_workspace_size(100, 60, 70, 80, 90, 1, 0, ctypes.byref(ws)) == 0
    up = lambda b: (b + 255) // 256 * 256
    assert ws.value == up(100 * 60 * 4) + up(60 * 80 * 4)
    # tensor-core forms: packed A, B^T, D^T, C, E (row operand) and F^T (column operand)
    assert L.ln_3mm_workspace_size(256, 256, 256, 256, 256, 1, 2, ctypes.byref(ws)) == 0
    tile = 2 * 16384  # two split terms of a 128 x 64 tile
    expect = tile * (2 * 4 + 2 * 4 + 2 * 4 + 2 * 4 + 2 * 4 + 2 * 4)
    assert ws.value == expect


def test_3mm_bwd_validation(L):
    F = [0x7F0000000000 + i * 0x100000 for i in range(9)]
    ws = ctypes.c_size_t(0)
    assert L.ln_3mm_bwd(4, 4, 4, 4, 4, *(P(x) for x in F[:5]), None, P(F[6]), P(F[7]), P(F[8]), None, 0, 1, 2,
                        None) == 1
    # dB aliasing dA, and dD aliasing the upstream gradient
    assert L.ln_3mm_bwd(8, 8, 8, 8, 8, *(P(x) for x in F[:5]), P(F[5]), P(F[5] + 64), P(F[7]), P(F[8]), None, 0,
                        1, 2, None) == 2
    assert L.ln_3mm_bwd(8, 8, 8, 8, 8, *(P(x) for x in F[:5]), P(F[5]), P(F[6]), P(F[7]), P(F[4]), None, 0, 1, 2,
                        None) == 2
    assert L.ln_3mm_bwd_workspace_size(100, 60, 70, 80, 90, 1, 0, ctypes.byref(ws)) == 0
    up = lambda b: (b + 255) // 256 * 256
    assert ws.value == 2 * (up(100 * 60 * 4) + up(60 * 80 * 4))


def test_gramschmidt_validation(L):
    FA, FQ, FR = 0x7F0000000000, 0x7F0000100000, 0x7F0000200000
    # negative size, unknown form, NULL operand, leading dimension below n
    assert L.ln_gramschmidt(-1, 4, P(FA), 4, P(FQ), 4, P(FR), 4, 1, None) == 1
    assert L.ln_gramschmidt(4, 4, P(FA), 4, P(FQ), 4, P(FR), 4, 5, None) == 1
    assert L.ln_gramschmidt(4, 4, P(FA), 4, P(FQ), 4, None, 4, 1, None) == 1
    assert "NULL" in last(L)
    assert L.ln_gramschmidt(4, 4, P(FA), 3, P(FQ), 4, P(FR), 4, 1, None) == 1
    # Q overlapping A other than exactly in place, R overlapping Q
    assert L.ln_gramschmidt(8, 8, P(FA), 8, P(FA + 64), 8, P(FR), 8, 1, None) == 2
    assert L.ln_gramschmidt(8, 8, P(FA), 8, P(FA), 9, P(FR), 8, 0, None) == 2
    assert L.ln_gramschmidt(8, 8, P(FA), 8, P(FQ), 8, P(FQ + 32), 8, 1, None) == 2
    # n == 0 is a no-op
    assert L.ln_gramschmidt(5, 0, None, 0, None, 0, None, 0, 1, None) == 0
    # tuning knob
    v = ctypes.c_int(0)
    assert L.ln_get_tuning(b"gs_rows", ctypes.byref(v)) == 0 and v.value == 4
    assert L.ln_set_tuning(b"gs_rows", 3) == 1
    assert L.ln_get_tuning(b"stream_k", ctypes.byref(v)) == 0 and v.value == 2
    assert L.ln_set_tuning(b"stream_k", 3) == 1
    assert L.ln_get_tuning(b"pair", ctypes.byref(v)) == 0 and v.value == 1
    assert L.ln_set_tuning(b"pair", 3) == 1
    assert L.ln_get_tuning(b"stage_beta", ctypes.byref(v)) == 0 and v.value == 1
    assert L.ln_set_tuning(b"stage_beta", 2) == 1
    assert L.ln_get_tuning(b"simt_exact", ctypes.byref(v)) == 0 and v.value == 1
    assert L.ln_set_tuning(b"simt_exact", 2) == 1
    assert L.ln_get_tuning(b"sym_wide", ctypes.byref(v)) == 0 and v.value == 0
    assert L.ln_set_tuning(b"sym_wide", 3) == 1
    assert L.ln_get_tuning(b"stage_out", ctypes.byref(v)) == 0 and v.value == 1
    assert L.ln_set_tuning(b"stage_out", 2) == 1
    assert L.ln_get_tuning(b"simt_tile", ctypes.byref(v)) == 0 and v.value == 0
    # launch timing modes: 0 off, 1 every launch, 2 spans
    assert L.ln_timing_enable(3) == 1 and L.ln_timing_enable(-1) == 1
    assert L.ln_timing_enable(2) == 0 and L.ln_timing_enable(0) == 0
    # peak probes: bad arguments are refused before anything is launched
    w = ctypes.c_double(1.0)
    probe = L.ln_peak_probe
    probe.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                      ctypes.c_void_p, ctypes.c_void_p]
    assert probe(9, 1, None, None, 0, ctypes.byref(w), None) == 1 and w.value == 0.0
    assert probe(0, 0, None, ctypes.c_void_p(256), 4, ctypes.byref(w), None) == 1  # iters < 1
    assert probe(1, 1 << 21, None, ctypes.c_void_p(256), 4, ctypes.byref(w), None) == 1  # iters > 2^20
    assert probe(0, 8, None, None, 4, ctypes.byref(w), None) == 1  # no error word
    assert probe(2, 8, None, ctypes.c_void_p(258), 4, ctypes.byref(w), None) == 1  # unaligned sink
    assert probe(3, 0, ctypes.c_void_p(256), ctypes.c_void_p(512), 24, ctypes.byref(w), None) == 1  # not x16
    assert probe(3, 0, ctypes.c_void_p(256), ctypes.c_void_p(272), 64, ctypes.byref(w), None) == 2  # overlap
    assert probe(3, 0, None, None, 0, None, None) == 1  # NULL work
    assert L.ln_set_tuning(b"simt_tile", 32) == 1 and L.ln_set_tuning(b"simt_tile", 1) == 1
