"""Planted slips in the oracle (CPU only) must fail the pins.

Each mutant replaces one oracle function with a plausible wrong version for the
duration of one test and checks that a pin of tests/test_oracle_pins.py notices.
"""
import math

import numpy as np
import pytest

import synth
from oracle import brute
from oracle import ustat_oracle as uo


def _brute_mismatch():
    g = synth.Graph(4, [(0, 1, 0), (2, 1, 2), (2, 3, 0), (3, 0, 2), (0, 2, 0)], [(1, 1)])
    n = 6
    rng = np.random.default_rng(4)
    facs = [synth.Factor(uo.MATRIX, data=rng.standard_normal((n, n))),
            synth.Factor(uo.VECTOR, data=rng.standard_normal(n)),
            synth.Factor(uo.MATRIX, data=rng.uniform(0.5, 1.5, (n, n)))]
    X = np.zeros((n, 1))
    r = uo.ustat(g, facs, X)
    b = brute.brute_all(g, facs, X)
    scale = max(abs(v) for v in b["V"])
    return abs(r["U_sum"] - b["U_sum"]) > 1e-9 * scale or any(
        abs(x - y) > 1e-9 * scale for x, y in zip(r["V"], b["V"]))


def _stirling_fails():
    parts = uo.set_partitions(4)
    return any(sum(uo.mu_closed_form(r) * n ** (max(r) + 1) for r in parts) != uo.falling_factorial(n, 4)
               for n in range(4, 12))


def test_mutant_mu_sign(monkeypatch):
    def bad(rgs):
        bl = uo.blocks(rgs)
        return math.prod(math.factorial(len(c) - 1) for c in bl)  # sign dropped
    monkeypatch.setattr(uo, "mu_closed_form", bad)
    assert _stirling_fails() and _brute_mismatch()


def test_mutant_mu_factorial(monkeypatch):
    def bad(rgs):
        bl = uo.blocks(rgs)
        sign = -1 if (len(rgs) - len(bl)) % 2 else 1
        return sign * math.prod(math.factorial(len(c)) for c in bl)  # (|C|)! instead of (|C|-1)!
    monkeypatch.setattr(uo, "mu_closed_form", bad)
    assert _stirling_fails()


def test_mutant_transposed_operand(monkeypatch):
    orig = uo._sum_out

    def bad(v, group):
        ax, arr = orig(v, group)
        return ax, (arr.T if arr.ndim == 2 else arr)   # result of a matrix step transposed
    monkeypatch.setattr(uo, "_sum_out", bad)
    assert _brute_mismatch()


def test_mutant_diagonal_dropped(monkeypatch):
    orig = uo._canonical

    def bad(axes, arr):
        if len(set(axes)) < len(axes):
            return (axes[0],), np.ones(np.asarray(arr).shape[0])   # intra-block factor ignored
        return orig(axes, arr)
    monkeypatch.setattr(uo, "_canonical", bad)
    assert _brute_mismatch()


def test_mutant_missing_partition(monkeypatch):
    orig = uo.set_partitions
    monkeypatch.setattr(uo, "set_partitions", lambda m: orig(m)[:-1])
    assert len(uo.set_partitions(4)) != 15 and _brute_mismatch()


def test_mutant_sparsify_keeps_diagonal(monkeypatch):
    monkeypatch.setattr(uo, "sparsify", lambda T: T)
    X = synth.normal_X(20, 3, 1)
    K = uo.factor_tensor(uo.RBF, X, 6.0)
    Kt = K - np.diag(np.diag(K))
    want = np.trace(Kt @ Kt @ Kt)
    got = uo.ustat(synth.triangle_graph(), [synth.rbf(3)], X, sparse=True)["U_sum"]
    assert got != pytest.approx(want, rel=1e-6)


def test_mutant_rbf_bandwidth(monkeypatch):
    orig = uo.factor_tensor

    def bad(kind, X, param=1.0, data=None):
        return orig(kind, X, param * 0.5 if kind == uo.RBF else param, data)
    monkeypatch.setattr(uo, "factor_tensor", bad)
    X = np.array([[0.0, 0.0], [1.0, 1.0]])
    assert uo.factor_tensor(uo.RBF, X, 4.0)[0, 1] != pytest.approx(math.exp(-0.5))
