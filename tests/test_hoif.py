"""HOIF chain U-statistics (Section 4.1): U(h_j) for the chain kernels
h_j = g g ... g f of the paper's equation for the HOIF kernel.

CPU: the binding's factor matrices against the definitions of g and f; the
oracle's U_sum against brute force over ordered distinct tuples; every V_pi of
the oracle against the closed form for rank-one factors (each pairwise factor
l_e(a) r_e(b): V_pi = prod over blocks of sum_i prod of the block's endpoint
vectors).  GPU: every chain order at n = 200 (two tiles, ragged tail) against
the oracle element by element, and order 5 at the paper's n = 10000 on sampled
low-treewidth partitions."""
import itertools
import math

import numpy as np
import pytest

import synth
from oracle import ustat_oracle as uo


def _factors(j, G, F):
    M = synth.MATRIX
    return [synth.Factor(M, 1.0, F)] if j == 2 else [synth.Factor(M, 1.0, G), synth.Factor(M, 1.0, F)]


def _gf(phi, A, Y):
    """g and f of the paper's HOIF kernel as matrices, from their definitions."""
    Psi, Theta = A[:, None] * phi, phi * Y[:, None]
    return Psi @ Psi.T, Psi @ Theta.T


def test_factor_matrices_follow_the_definitions():
    pytest.importorskip("torch")
    from paper_2508_12627_gb300 import hoif
    phi, A, Y = synth.hoif_sample(40, k=5, seed=3)
    G, F = hoif.factor_matrices(phi, A, Y)
    # the device factors' data: Psi and [Psi | Theta], whose products (the
    # oracle's GRAM and LOWRANK definitions) are g and f
    TG, TF = hoif.factor_terms(phi, A, Y)
    assert TG.shape == (40, 5) and TF.shape == (40, 10)
    assert np.allclose(uo.factor_tensor(uo.GRAM, np.zeros((40, 1)), 5, TG), G, rtol=1e-13, atol=1e-13)
    assert np.allclose(uo.factor_tensor(uo.LOWRANK, np.zeros((40, 1)), 5, TF), F, rtol=1e-13, atol=1e-13)
    for a, b in [(0, 1), (3, 3), (7, 2), (39, 11)]:
        assert abs(G[a, b] - A[a] * A[b] * phi[a] @ phi[b]) <= 1e-12 * (1 + abs(G[a, b]))
        assert abs(F[a, b] - A[a] * (phi[a] @ phi[b]) * Y[b]) <= 1e-12 * (1 + abs(F[a, b]))
    for j in range(2, 8):
        g, names = hoif.chain_graph(j)
        assert g.edges == synth.hoif_chain_graph(j).edges and len(names) == (1 if j == 2 else 2)


@pytest.mark.parametrize("j", [2, 3, 4, 5, 6, 7])
def test_oracle_chain_against_brute_force(j):
    n = 8
    phi, A, Y = synth.hoif_sample(n, k=3, seed=j)
    Psi, Theta = A[:, None] * phi, phi * Y[:, None]
    G, F = Psi @ Psi.T, Psi @ Theta.T
    r = uo.ustat(synth.hoif_chain_graph(j), _factors(j, G, F), np.zeros((n, 1)))
    # the partition sum's rounding scale: sum |mu| V_pi over |factors|
    a = uo.ustat(synth.hoif_chain_graph(j), _factors(j, G, F), np.zeros((n, 1)), absolute=True)
    uabs = float(np.abs(np.asarray(a["mu"], dtype=float)) @ np.asarray(a["V"]))
    terms = []
    for t in itertools.permutations(range(n), j):
        v = F[t[j - 2], t[j - 1]]
        for s in range(j - 2):
            v *= G[t[s], t[s + 1]]
        terms.append(v)
    assert abs(r["U_sum"] - math.fsum(terms)) <= 1e-13 * uabs


@pytest.mark.parametrize("j", [3, 5, 7])
def test_oracle_rank_one_closed_form(j):
    # k = 1: g = psi psi', f = psi theta'.  Vertex v of the chain carries psi once
    # per edge it starts (and per g edge it ends), theta at the end vertex.
    n = 9
    phi, A, Y = synth.hoif_sample(n, k=1, seed=10 + j)
    psi, theta = A * phi[:, 0], phi[:, 0] * Y
    G, F = np.outer(psi, psi), np.outer(psi, theta)
    r = uo.ustat(synth.hoif_chain_graph(j), _factors(j, G, F), np.zeros((n, 1)))
    w = [psi ** (1 if v == 0 else 2) for v in range(j - 1)] + [theta]   # per chain vertex
    for rgs, V in zip(r["rgs"], r["V"]):
        want = 1.0
        for blk in range(max(rgs) + 1):
            prod = np.ones(n)
            for v in range(j):
                if rgs[v] == blk:
                    prod = prod * w[v]
            want *= prod.sum()
        scale = 1.0
        for blk in range(max(rgs) + 1):
            prod = np.ones(n)
            for v in range(j):
                if rgs[v] == blk:
                    prod = prod * np.abs(w[v])
            scale *= prod.sum()
        assert abs(V - want) <= 1e-12 * scale, (rgs, V, want)


# ---------------------------------------------------------------- GPU

TOL = {"fp64": 1e-11, "bf16x4": 1e-8, "bf16x3": 1e-6}


@pytest.fixture(scope="module")
def small():
    n = 200
    phi, A, Y = synth.hoif_sample(n, seed=0)
    G, F = _gf(phi, A, Y)
    ref = {}
    for j in range(2, 8):
        fs = _factors(j, G, F)
        g = synth.hoif_chain_graph(j)
        ref[j] = (uo.ustat(g, fs, np.zeros((n, 1))), uo.ustat(g, fs, np.zeros((n, 1)), absolute=True))
    return (phi, A, Y), ref


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "bf16x4", "bf16x3"])
def test_hoif_chains_against_oracle(small, precision):
    from paper_2508_12627_gb300 import build
    build.build()
    from paper_2508_12627_gb300 import hoif
    (phi, A, Y), ref = small
    hc = hoif.HoifChains(200, precision=precision)
    hc.ws.fill_(255)                                            # NaN bytes: no stale reads
    got = hc.evaluate(phi, A, Y)
    tol = TOL[precision]
    for j in range(2, 8):
        r, ra = ref[j]
        V = hc.out[j][2:].cpu().numpy()
        Vabs = np.maximum(np.asarray(ra["V"]), 1e-300)
        err = np.abs(V - np.asarray(r["V"])) / Vabs
        assert err.max() <= tol, (precision, j, err.max(), int(err.argmax()))
        uabs = float(np.abs(np.asarray(ra["mu"], dtype=float)) @ np.asarray(ra["V"]))
        assert abs(got[j] - r["U_sum"]) <= tol * uabs, (precision, j)


@pytest.mark.gpu
def test_hoif_order5_full_size_sampled_partitions():
    # n = 10000 (the largest n of the paper's HOIF table) in bf16x4; the oracle
    # evaluates four partitions of treewidth <= 1 (n^2 work each)
    from paper_2508_12627_gb300 import build
    build.build()
    from paper_2508_12627_gb300 import hoif
    n, j = 10000, 5
    phi, A, Y = synth.hoif_sample(n, seed=1)
    hc = hoif.HoifChains(n, orders=(j,), precision="bf16x4")
    hc.evaluate(phi, A, Y)
    V = hc.out[j][2:].cpu().numpy()
    G, F = _gf(phi, A, Y)
    g = synth.hoif_chain_graph(j)
    parts = uo.set_partitions(j)
    tw = [uo.treewidth_bruteforce(max(r) + 1, uo.quotient_edges(g, r)) for r in parts]
    low = [i for i, t in enumerate(tw) if t <= 1]
    pick = [low[0], low[len(low) // 3], low[2 * len(low) // 3], low[-1]]
    sel = [parts[i] for i in pick]
    fs = _factors(j, G, F)
    ref = uo.ustat(g, fs, np.zeros((n, 1)), partitions=sel)
    absref = uo.ustat(g, fs, np.zeros((n, 1)), partitions=sel, absolute=True)
    for k, i in enumerate(pick):
        assert abs(V[i] - ref["V"][k]) <= 1e-8 * absref["V"][k], (parts[i], V[i], ref["V"][k])
