"""Squared distance covariance (Section 4.3) as four exact U-statistics.

CPU: the oracle's four U_sums, combined with the engine binding's coefficients,
equal brute force over the paper's order-4 kernel and the U-centred closed form
(a different derivation: the unbiased estimator as an inner product of
U-centred distance matrices); special cases.  GPU: the engine at the paper's
n = 138 on the synthetic sector returns, term by term against the oracle and as
dCov^2 against the closed form, in FP64 and the split modes."""
import itertools
import math

import numpy as np
import pytest

import synth
from oracle import ustat_oracle as uo


def _dist(Z):
    Z = np.asarray(Z, dtype=np.float64)
    return np.sqrt(((Z[:, None, :] - Z[None, :, :]) ** 2).sum(-1))


def u_centred(a, b):
    """The U-centred estimator: (1 / (n (n - 3))) sum_{i != j} A~_ij B~_ij."""
    n = a.shape[0]

    def uc(d):
        r = d.sum(1)
        t = d.sum()
        D = d - r[:, None] / (n - 2) - r[None, :] / (n - 2) + t / ((n - 1) * (n - 2))
        np.fill_diagonal(D, 0.0)
        return D

    return float((uc(a) * uc(b)).sum() / (n * (n - 3)))


def brute(a, b):
    n = a.shape[0]
    s = math.fsum(a[i, j] * (b[k, l] + b[i, j] - b[i, k] - b[j, l])
                  for i, j, k, l in itertools.permutations(range(n), 4))
    return s / math.perm(n, 4)


def oracle_terms(a, b):
    from paper_2508_12627_gb300 import dcov
    n = a.shape[0]
    F = [synth.Factor(synth.MATRIX, 1.0, a), synth.Factor(synth.MATRIX, 1.0, b)]
    us_ = [uo.ustat(synth.Graph(k, e), F, np.zeros((n, 1)))["U_sum"] for _, k, e in dcov.TERMS]
    coef = [c(n) for c, _, _ in dcov.TERMS]
    return us_, coef


@pytest.mark.parametrize("n,seed", [(7, 0), (10, 1), (12, 2)])
def test_terms_give_the_papers_kernel_and_the_closed_form(n, seed):
    pytest.importorskip("torch")
    rng = np.random.default_rng(seed)
    a, b = _dist(rng.standard_normal((n, 3))), _dist(rng.standard_t(3, (n, 2)))
    us_, coef = oracle_terms(a, b)
    d = math.fsum(c * u for c, u in zip(coef, us_)) / math.perm(n, 4)
    assert abs(d - brute(a, b)) <= 1e-12 * abs(d)
    assert abs(d - u_centred(a, b)) <= 1e-12 * abs(d)


def test_special_cases():
    pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    X = rng.standard_normal((9, 2))
    a = _dist(X)
    us_, coef = oracle_terms(a, np.zeros_like(a))          # Y constant: no dependence at all
    assert math.fsum(c * u for c, u in zip(coef, us_)) == 0.0
    us_, coef = oracle_terms(a, a)                           # dCov^2(X, X) = dVar^2 > 0
    assert math.fsum(c * u for c, u in zip(coef, us_)) > 0.0
    # a rigid motion of X leaves every distance, so dCov^2, unchanged
    Q, _ = np.linalg.qr(rng.standard_normal((2, 2)))
    b = _dist(rng.standard_normal((9, 1)))
    assert abs(u_centred(_dist(X @ Q.T + 3.0), b) - u_centred(a, b)) <= 1e-12 * abs(u_centred(a, b))


def test_binding_distances_follow_the_definition():
    pytest.importorskip("torch")
    from paper_2508_12627_gb300 import dcov
    rng = np.random.default_rng(5)
    for n, p in [(138, 40), (700, 60)]:                          # one block, several blocks of rows
        Z = rng.standard_normal((n, p))
        D = dcov.distances(Z)
        assert np.max(np.abs(D - _dist(Z))) <= 1e-13 * np.max(D) and np.array_equal(D, D.T)
    assert np.array_equal(dcov.distances(np.arange(5.0)), np.abs(np.subtract.outer(np.arange(5.0), np.arange(5.0))))


def test_sector_returns_shape():
    R = synth.sector_returns()
    assert len(R) == 11 and all(r.shape[0] == 138 and 20 <= r.shape[1] <= 70 for r in R)


@pytest.mark.gpu
# the parity suite's bounds below the full sample sizes: float64 storage (fp64,
# bf16x4) to 1e-12 and 1e-8, float32 storage (bf16x3) to 5e-7
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("bf16x4", 1e-8), ("bf16x3", 5e-7)])
def test_dcov_at_n_138_against_oracle_and_closed_form(precision, tol):
    from paper_2508_12627_gb300 import build
    build.build()
    from paper_2508_12627_gb300 import dcov
    R = synth.sector_returns()
    dc = dcov.DCov2(138, precision=precision)
    for i, j in [(0, 1), (3, 7), (10, 5)]:
        a, b = _dist(R[i]), _dist(R[j])
        dc.ws.fill_(255)                                     # NaN bytes: no stale reads
        val, scale = dc.evaluate(R[i], R[j])
        ref_terms, coef = oracle_terms(a, b)
        got_terms = [float(o[0].item()) for o in dc.out]
        for g, r in zip(got_terms, ref_terms):               # every term is a sum of positive products
            assert abs(g - r) <= tol * abs(r), (precision, i, j, g, r)
        assert abs(val - u_centred(a, b)) <= tol * scale, (precision, i, j, val, u_centred(a, b), scale)


@pytest.mark.gpu
def test_dcov_graph_replay_matches_eager():
    # the distance matrices of three samples and the evaluations of two pairs,
    # captured into one CUDA graph: a replay on new sample contents gives what the
    # eager launches give on them
    import torch
    from paper_2508_12627_gb300 import build
    build.build()
    from paper_2508_12627_gb300 import dcov
    R = synth.sector_returns()
    n = R[0].shape[0]
    dc = dcov.DCov2(n)
    Z = [torch.from_numpy(np.ascontiguousarray(R[i], dtype=np.float64)).cuda() for i in (0, 4, 9)]
    D = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in Z]
    outs = [[torch.empty_like(o) for o in dc.out] for _ in range(2)]

    def enqueue():
        for z, d in zip(Z, D):
            dc.distance(z, d)
        dc.launch_matrices(D[0], D[1], outs[0])
        dc.launch_matrices(D[2], D[0], outs[1])

    graph = dc.capture(enqueue)
    # new contents of the same shapes: the rows in reverse order, rescaled
    new = [np.ascontiguousarray(R[i][::-1] * 1.5, dtype=np.float64) for i in (0, 4, 9)]
    for z, v in zip(Z, new):
        z.copy_(torch.from_numpy(v))
    graph.replay()
    torch.cuda.synchronize()
    got = [[float(x[0].item()) for x in o] for o in outs]
    enqueue()
    torch.cuda.synchronize()
    want = [[float(x[0].item()) for x in o] for o in outs]
    for g, w in zip(got, want):
        assert g == pytest.approx(w, rel=1e-13, abs=0.0)
    # and the replayed values are those of the new samples
    a, b = _dist(new[0]), _dist(new[1])
    ref_terms, _ = oracle_terms(a, b)
    for g, r in zip(got[0], ref_terms):
        assert abs(g - r) <= 1e-12 * abs(r)


def test_planted_coefficient_mistakes_fail_the_pins():
    pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    n = 9
    a, b = _dist(rng.standard_normal((n, 2))), _dist(rng.standard_normal((n, 2)))
    us_, coef = oracle_terms(a, b)
    want = brute(a, b)
    good = math.fsum(c * u for c, u in zip(coef, us_)) / math.perm(n, 4)
    assert abs(good - want) <= 1e-12 * abs(want)
    for bad in ([coef[0], coef[1] / (n - 3), coef[2], coef[3]],      # (n - 2) instead of (n - 2)(n - 3)
                [coef[0], coef[1], coef[2] * (n - 2) / (n - 3), coef[3]],
                [coef[0], coef[1], coef[2], -coef[3]]):
        d = math.fsum(c * u for c, u in zip(bad, us_)) / math.perm(n, 4)
        assert abs(d - want) > 1e-6 * abs(want)
