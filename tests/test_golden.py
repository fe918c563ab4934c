"""Hand-derived examples (tests/golden/hand_examples.json) against the oracle."""
import json
import os
from fractions import Fraction

import numpy as np

import oracle

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")))


def a(x):
    return np.asarray(x, dtype=np.float64)


def test_golden_oracle():
    g = G["gemm"]
    assert np.array_equal(oracle.gemm(a(g["A"]), a(g["B"]), a(g["C"]), g["alpha"], g["beta"]), a(g["out"]))
    g = G["chain"]
    E, F = oracle.gemm_chain(a(g["A"]), a(g["B"]), a(g["C"]), a(g["D"]), g["alpha"], g["beta"])
    assert np.array_equal(E, a(g["E"])) and np.array_equal(F, a(g["F"]))
    assert np.array_equal(oracle.covariance(a(G["covariance"]["X"])), a(G["covariance"]["out"]))
    # sqrt(8)*sqrt(8) is 8 only to within one rounding, hence the 1e-15 tolerance
    assert np.max(np.abs(oracle.correlation(a(G["correlation"]["X"])) - a(G["correlation"]["out"]))) < 1e-15
    g = G["syrk"]
    assert np.array_equal(oracle.syrk(a(g["A"]), a(g["C"]), g["alpha"], g["beta"], g["fill"]), a(g["out"]))
    g = G["syr2k"]
    assert np.array_equal(oracle.syr2k(a(g["A"]), a(g["B"]), a(g["C"]), g["alpha"], g["beta"], g["fill"]), a(g["out"]))


def test_golden_gramschmidt_oracle():
    g = G["gramschmidt"]
    Q, R = oracle.gramschmidt(a(g["A"]))
    Qe = np.array([[float(Fraction(x)) for x in row] for row in g["Q"]])
    Re = np.array([[float(Fraction(x)) for x in row] for row in g["R"]])
    # one division and a square root per entry: within a few FP64 roundings
    assert np.max(np.abs(Q - Qe)) < 1e-15 and np.max(np.abs(R - Re)) < 1e-14
