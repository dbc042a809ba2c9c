"""Pins of the FP64 oracle to things other than itself: values the paper prints,
closed forms, textbook identities, and brute force on tiny inputs.

Each test names the passage it follows.  A plausible slip in the oracle (a dropped
factor, a wrong Moebius sign, a transposed operand, a wrong diagonal, a missed
partition) fails at least one of them; tests/test_oracle_mutants.py plants such
slips and checks that they are caught.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import brute
from oracle import ustat_oracle as uo
from tests.conftest import GOLDEN


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _rgs_from_blocks(blocks_1based, m):
    lab = [None] * m
    for j, b in enumerate(sorted((sorted(b) for b in blocks_1based), key=lambda b: b[0])):
        for i in b:
            lab[i - 1] = j
    return tuple(lab)


# ---------------------------------------------------------------- partitions and mu

def test_bell_numbers():
    # Table 'HOIF' (Appendix H), "V-stat terms (Bell number)" column, m = 2..9
    g = _golden("hoif_chain_table.json")
    for m, bell in zip(g["m"], g["bell"]):
        if m <= 9:
            assert len(uo.set_partitions(m)) == bell


def test_rgs_lexicographic_and_distinct():
    for m in range(1, 7):
        p = uo.set_partitions(m)
        assert p == sorted(p)
        assert len(set(p)) == len(p)
        for rgs in p:
            assert rgs[0] == 0
            assert all(rgs[i] <= max(rgs[:i]) + 1 for i in range(1, m))


def test_mu_closed_form_equals_lattice_recursion():
    # Lemma 'Decomposition of U into V' (Section 3.3) vs Definition 'Moebius Function'
    # applied to the partition lattice (Appendix E).
    for m in range(1, 6):
        lat = uo.mobius_lattice(m)
        finest = tuple(range(m))
        for rgs in uo.set_partitions(m):
            assert lat[(finest, rgs)] == uo.mu_closed_form(rgs)


def test_extended_mobius_formula():
    # Lemma 'ext_decomp_u_to_v' (Appendix E): mu(pi, rho) = (-1)^(|pi|-|rho|) prod (kappa-1)!
    m = 4
    lat = uo.mobius_lattice(m)
    for (pi, rho), val in lat.items():
        bl_pi = uo.blocks(pi)
        kappas = [sum(1 for q in bl_pi if rho[q[0]] == j) for j in range(max(rho) + 1)]
        sign = -1 if ((max(pi) + 1) - (max(rho) + 1)) % 2 else 1
        assert val == sign * math.prod(math.factorial(k - 1) for k in kappas)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7])
def test_sum_mu_n_pow_blocks_is_falling_factorial(m):
    # The constant kernel h = 1 has V_pi = n^|pi| and U = (n)_m (Definition
    # 'U-Statistic'); with Lemma 'Decomposition of U into V' this is the signed
    # Stirling identity sum_pi mu_pi n^|pi| = n (n-1) ... (n-m+1).
    parts = uo.set_partitions(m)
    for n in [m, m + 1, 10, 37]:
        s = sum(uo.mu_closed_form(r) * n ** (max(r) + 1) for r in parts)
        assert s == uo.falling_factorial(n, m)


def test_stirling_m4_polynomial():
    parts = uo.set_partitions(4)
    for n in range(4, 30):
        s = sum(uo.mu_closed_form(r) * n ** (max(r) + 1) for r in parts)
        assert s == n ** 4 - 6 * n ** 3 + 11 * n ** 2 - 6 * n


# ---------------------------------------------------------------- notation and sparsification

def test_induced_notation_example():
    # Example 'A_pi' (Section 3.3)
    g = _golden("path4_examples.json")
    sig = [(tuple(i - 1 for i in t), 0) for t in g["signature"]]
    rgs = _rgs_from_blocks(g["induced_example"]["partition"], 4)
    ind = uo.induced_notation(sig, rgs)
    want = [tuple(i - 1 for i in t) for t in g["induced_example"]["induced"]]
    assert [t for t, _ in ind] == want


def test_path4_sparsification_survivors():
    # Example 'sparsification' (Section 3.3): exactly five partitions survive
    g = _golden("path4_examples.json")
    sig = uo.signature(synth.path(4))
    got = {r for r in uo.set_partitions(4) if uo.survives(sig, r)}
    want = {_rgs_from_blocks(b, 4) for b in g["survivors"]}
    assert got == want


def test_chain_sparsified_counts():
    # Table 'HOIF' (Appendix H), "V-stat terms (sparsification)" column
    g = _golden("hoif_chain_table.json")
    for m, cnt in zip(g["m"], g["sparsified"]):
        if m > 9:
            continue
        sig = uo.signature(synth.path(m))
        assert sum(uo.survives(sig, r) for r in uo.set_partitions(m)) == cnt


def test_complete_graph_only_finest_survives():
    # Appendix I: for the K_m signature only the finest partition survives
    for m in range(2, 7):
        sig = uo.signature(synth.complete(m))
        surv = [r for r in uo.set_partitions(m) if uo.survives(sig, r)]
        assert surv == [tuple(range(m))]


# ---------------------------------------------------------------- treewidth pins

def test_cycle4_treewidth():
    # Example 'treewidth' (Section 2.3)
    assert uo.treewidth_bruteforce(4, [(0, 1), (1, 2), (2, 3), (3, 0)]) == \
        _golden("path4_examples.json")["cycle4_treewidth"]


def test_path4_quotient_treewidths():
    # Example 'U_complexity' (Section 3.3): M = 2, N1 = 4, N2 = 1
    g = synth.path(4)
    sig = uo.signature(g)
    tws = [uo.treewidth_bruteforce(max(r) + 1, uo.quotient_edges(g, r))
           for r in uo.set_partitions(4) if uo.survives(sig, r)]
    want = _golden("path4_examples.json")["survivor_treewidth"]
    assert max(tws) == want["M"] and tws.count(1) == want["N1"] and tws.count(2) == want["N2"]


def _canon(k, edges):
    best = None
    for p in itertools.permutations(range(k)):
        e = tuple(sorted(tuple(sorted((p[a], p[b]))) for a, b in edges))
        best = e if best is None or e < best else best
    return (k, best)


def test_path4_quotient_isomorphism_types():
    # Example 'quotient' (Section 2.3): 15 partitions, 5 isomorphism types
    g = synth.path(4)
    types = {_canon(max(r) + 1, uo.quotient_edges(g, r)) for r in uo.set_partitions(4)}
    assert len(types) == _golden("path4_examples.json")["quotient_isomorphism_types"]


@pytest.mark.parametrize("m", [4, 5, 6, 7])
def test_chain_N_l_counts(m):
    # Table 'HOIF_Nl' (Appendix H), dp rows: exact quotient treewidth counts, and
    # Table 'HOIF' column M.
    g = synth.path(m)
    sig = uo.signature(g)
    counts = [0, 0, 0, 0]
    for r in uo.set_partitions(m):
        if uo.survives(sig, r):
            tw = uo.treewidth_bruteforce(max(r) + 1, uo.quotient_edges(g, r))
            counts[tw - 1] += 1
    gold = _golden("hoif_chain_table.json")
    assert counts == gold["N_l_dp"][str(m)]
    assert max(l + 1 for l, c in enumerate(counts) if c) == gold["M"][gold["m"].index(m)]


def test_max_treewidth_by_edges_small_graphs():
    # Observation 'treewidth_table' (Appendix F) for e <= 10: the maximum is reached
    # by graphs on at most 5 vertices (K_5 has 10 edges), so enumerate those.
    gold = _golden("max_treewidth_by_edges.json")
    allpairs = [(a, b) for a in range(5) for b in range(a + 1, 5)]
    best = {}
    for e in range(1, 11):
        best[e] = max(uo.treewidth_bruteforce(5, list(es)) for es in itertools.combinations(allpairs, e))
    for e, t in zip(gold["e"], gold["t"]):
        if e <= 10:
            assert best[e] == t, (e, best[e], t)


# ---------------------------------------------------------------- kernel maps

def test_kernel_maps_by_hand():
    X = np.array([[0.0, 0.0], [1.0, 1.0], [2.0, -1.0]])
    K = uo.factor_tensor(uo.RBF, X, 4.0)
    assert np.allclose(np.diag(K), 1.0) and np.array_equal(K, K.T)
    assert K[0, 1] == pytest.approx(math.exp(-2.0 / 4.0), rel=1e-15)
    assert K[1, 2] == pytest.approx(math.exp(-5.0 / 4.0), rel=1e-15)
    L = uo.factor_tensor(uo.LINEAR, X, 2.0)
    assert L[1, 2] == pytest.approx(0.5) and L[2, 2] == pytest.approx(2.5)
    t = uo.factor_tensor(uo.TANH_DOT, X, data=np.array([0.5, 0.25]))
    assert t[2] == pytest.approx(math.tanh(0.75), rel=1e-15)


# ---------------------------------------------------------------- closed forms for U and V

def test_product_kernel_closed_form():
    # h(x1, x2) = x1 x2 (m = 2, d = 1): U = (sum x)^2 - sum x^2
    x = np.random.default_rng(3).standard_normal((50, 1))
    g = synth.Graph(2, [(0, 1, 0)], [])
    r = uo.ustat(g, [synth.Factor(uo.LINEAR, 1.0)], x)
    want = x.sum() ** 2 - (x ** 2).sum()
    assert r["U_sum"] == pytest.approx(want, rel=1e-12)
    assert r["U_mean"] == pytest.approx(want / (50 * 49), rel=1e-12)


@pytest.mark.parametrize("graph", [synth.triangle_graph(), synth.cycle4_graph(),
                                   synth.path5_chord_graph(), synth.k4_plus_cycle_graph()])
def test_constant_kernel(graph):
    # constant factors c: V_pi = c^|E| n^|pi| (times the unary constant), U = c^|E| (n)_m
    n, c = 7, 1.5
    facs = [synth.Factor(uo.MATRIX, data=np.full((n, n), c)), synth.Factor(uo.VECTOR, data=np.full(n, 2.0))]
    X = np.zeros((n, 1))
    r = uo.ustat(graph, facs, X)
    E, Un = len(graph.edges), len(graph.unary)
    for rgs, v in zip(r["rgs"], r["V"]):
        assert v == pytest.approx(c ** E * 2.0 ** Un * n ** (max(rgs) + 1), rel=1e-13)
    assert r["U_sum"] == pytest.approx(c ** E * 2.0 ** Un * uo.falling_factorial(n, graph.m), rel=1e-12)


@pytest.mark.parametrize("graph", [synth.triangle_graph(), synth.cycle4_graph(),
                                   synth.path5_chord_graph(), synth.k4_plus_cycle_graph(), synth.path(6)])
def test_rank1_integer_factors_exact(graph):
    # K = u u^T on every edge and the unary factor u: V_pi = prod_B p_{deg(B)}(u)
    # with p_k = sum_i u_i^k and deg(B) the number of factor slots landing in B.
    # Integer-valued, so the oracle must be exact.
    n = 23
    u = synth.ternary_vector(n, 5)
    facs = [synth.Factor(uo.MATRIX, data=np.outer(u, u)), synth.Factor(uo.VECTOR, data=u)]
    r = uo.ustat(graph, facs, np.zeros((n, 1)))
    for rgs, v in zip(r["rgs"], r["V"]):
        deg = [0] * (max(rgs) + 1)
        for a, b, _ in graph.edges:
            deg[rgs[a]] += 1
            deg[rgs[b]] += 1
        for a, _ in graph.unary:
            deg[rgs[a]] += 1
        want = math.prod(int(np.sum(u ** k)) for k in deg)
        assert v == want


def test_sparse_triangle_closed_form():
    # only the finest partition survives for K_3; U = tr(K~^3)
    X = synth.normal_X(40, 3, 7)
    f = [synth.rbf(3)]
    K = uo.factor_tensor(uo.RBF, X, 6.0)
    Kt = K.copy()
    np.fill_diagonal(Kt, 0)
    want = np.trace(Kt @ Kt @ Kt)
    for sparse in (True, False):
        assert uo.ustat(synth.triangle_graph(), f, X, sparse=sparse)["U_sum"] == pytest.approx(want, rel=1e-12)


def test_sparse_cycle4_closed_form():
    # U = tr(K~^4) - 2 sum_a (sum_b K~_ab^2)^2 + sum_ab K~_ab^4 (inclusion-exclusion over a=c, b=d)
    X = synth.normal_X(35, 4, 8)
    f = [synth.rbf(4)]
    K = uo.factor_tensor(uo.RBF, X, 8.0)
    Kt = K.copy()
    np.fill_diagonal(Kt, 0)
    K2 = Kt @ Kt
    want = np.trace(K2 @ K2) - 2 * np.sum(np.sum(Kt ** 2, axis=1) ** 2) + np.sum(Kt ** 4)
    for sparse in (True, False):
        assert uo.ustat(synth.cycle4_graph(), f, X, sparse=sparse)["U_sum"] == pytest.approx(want, rel=1e-11)


def test_motif_counts_complete_graph():
    # Appendix I: r_2 and r_8 on the complete graph K_n give C(n,3) and C(n,4)
    for case in _golden("motif_constants.json")["cases"]:
        n, m = case["n"], case["m"]
        A = np.ones((n, n)) - np.eye(n)
        r = uo.ustat(synth.complete(m), [synth.Factor(uo.MATRIX, data=A)], np.zeros((n, 1)), sparse=True)
        assert r["U_sum"] / case["inv_constant"] == pytest.approx(case["count"], abs=1e-9)
        assert math.comb(n, m) == case["count"]


# ---------------------------------------------------------------- brute force

def _asym_factors(n, seed):
    rng = np.random.default_rng(seed)
    return [synth.Factor(uo.MATRIX, data=rng.standard_normal((n, n))),
            synth.Factor(uo.VECTOR, data=rng.standard_normal(n)),
            synth.Factor(uo.MATRIX, data=rng.uniform(0.5, 1.5, (n, n)))]


BRUTE_GRAPHS = [
    synth.triangle_graph(), synth.cycle4_graph(), synth.path5_chord_graph(),
    synth.Graph(4, [(0, 1, 0), (2, 1, 2), (2, 3, 0), (3, 0, 2), (0, 2, 0)], [(1, 1)]),  # asymmetric, mixed orientation
    synth.Graph(5, [(0, 1, 0), (1, 0, 2), (1, 2, 0), (3, 4, 2)], [(2, 1), (4, 1)]),     # repeated pair, two components
    synth.k4_plus_cycle_graph(),
]


@pytest.mark.parametrize("gi", range(len(BRUTE_GRAPHS)))
def test_partition_sum_equals_brute_force(gi):
    # Algorithm 4 and the identity V_pi = Einsum(T, A_pi) against the definitions
    # (U over ordered distinct tuples; V_pi over the V-set), asymmetric factors.
    g = BRUTE_GRAPHS[gi]
    n = 7 if g.m <= 5 else 6
    facs = _asym_factors(n, gi)
    X = np.zeros((n, 1))
    r = uo.ustat(g, facs, X)
    b = brute.brute_all(g, facs, X)
    scale = max(abs(v) for v in b["V"])
    for v1, v2 in zip(r["V"], b["V"]):
        assert abs(v1 - v2) <= 1e-12 * scale
    assert abs(r["U_sum"] - b["U_sum"]) <= 1e-11 * scale
    rs = uo.ustat(g, facs, X, sparse=True)
    assert abs(rs["U_sum"] - b["U_sum"]) <= 1e-11 * scale


@pytest.mark.parametrize("gi", [1, 3, 4])
def test_v_is_sum_of_coarser_restricted_u(gi):
    # Lemma 'decomp_v_to_u' (Appendix E): V_pi = sum over rho >= pi of U_rho, with U_rho
    # the restricted U-statistic (Definition 'Restricted U-Statistic'), all by brute force
    g = BRUTE_GRAPHS[gi]
    n = 6
    facs = _asym_factors(n, 10 + gi)
    b = brute.brute_all(g, facs, np.zeros((n, 1)))
    parts = b["rgs"]
    scale = max(abs(v) for v in b["V"])
    for i, pi in enumerate(parts):
        s = sum(b["U_pattern"][j] for j, rho in enumerate(parts) if uo.refines(pi, rho))
        assert abs(s - b["V"][i]) <= 1e-12 * scale


def test_workload_graphs_against_brute_force():
    # the four workload graphs with their own kernel maps, tiny n
    for name in ["triangle_rbf", "c4_rbf", "path5_chord_linear_tanh", "k4_cycle_rbf"]:
        w = synth.workload(name, n=8 if name != "k4_cycle_rbf" else 6)
        r = uo.ustat(w.graph, w.factors, w.X)
        b = brute.brute_all(w.graph, w.factors, w.X)
        scale = max(abs(v) for v in b["V"])
        assert abs(r["U_sum"] - b["U_sum"]) <= 1e-12 * scale
        for v1, v2 in zip(r["V"], b["V"]):
            assert abs(v1 - v2) <= 1e-12 * scale


def test_triangle_workload_full_size_brute_force():
    # the triangle workload at its full size n = 200 (8e6 tuples)
    w = synth.workload("triangle_rbf")
    r = uo.ustat(w.graph, w.factors, w.X)
    b = brute.brute_all(w.graph, w.factors, w.X)
    assert r["U_sum"] == pytest.approx(b["U_sum"], rel=1e-12)
    for v1, v2 in zip(r["V"], b["V"]):
        assert v1 == pytest.approx(v2, rel=1e-12)


# ---------------------------------------------------------------- metamorphic

def test_row_permutation_invariance():
    w = synth.workload("c4_rbf", n=60)
    r1 = uo.ustat(w.graph, w.factors, w.X)
    perm = np.random.default_rng(0).permutation(60)
    r2 = uo.ustat(w.graph, w.factors, w.X[perm])
    for a, b in zip(r1["V"], r2["V"]):
        assert a == pytest.approx(b, rel=1e-12)


def test_elimination_order_independence():
    w = synth.workload("path5_chord_linear_tanh", n=30)
    sig = uo.signature(w.graph)
    T = uo.tensorize(w.graph, w.factors, w.X)
    rgs = tuple(range(5))
    ind = uo.induced_notation(sig, rgs)
    tens = [(t, T[f]) for t, f in ind]
    vals = [uo.einsum_eliminate(5, tens, list(o)) for o in itertools.permutations(range(5))]
    assert max(vals) - min(vals) <= 1e-11 * max(abs(v) for v in vals)


def test_n_equals_m_and_small_n():
    # n = m: U is the sum over the m! orderings of the whole sample
    w = synth.workload("c4_rbf", n=4)
    r = uo.ustat(w.graph, w.factors, w.X)
    b = brute.brute_all(w.graph, w.factors, w.X)
    assert r["U_sum"] == pytest.approx(b["U_sum"], rel=1e-12)
    # n < m: the U-statistic is an empty sum, and the Moebius sum also gives 0
    w = synth.workload("c4_rbf", n=3)
    r = uo.ustat(w.graph, w.factors, w.X)
    assert abs(r["U_sum"]) <= 1e-12 * max(abs(v) for v in r["V"])


def test_einsum_notation_sequence_of_k4():
    # Appendix D, the example after Definition "Einsum Notation Sequence": the
    # oracle's elimination of K4 under sigma = (1, 2, 3, 4) leaves exactly the
    # printed tuple lists, and its value is the full contraction
    g = _golden("einsum_sequence_k4.json")
    rng = np.random.default_rng(0)
    n = 5
    tens = [(tuple(v - 1 for v in t), rng.random((n, n))) for t in g["signature"]]
    trace = []
    val = uo.einsum_eliminate(4, tens, order=[v - 1 for v in g["sigma"]], trace=trace)
    want = [sorted(tuple(v - 1 for v in t) for t in step) for step in g["sequence"][1:]]
    assert trace == want
    full = np.einsum("ab,ac,ad,bc,bd,cd->", *[a for _, a in tens])
    assert abs(val - full) <= 1e-12 * abs(full)


def test_device_built_factor_kinds_by_hand():
    # DIST: points on a line at 0, 1, 3 -> |i - j|; points at the corners of a unit
    # square -> 1 and sqrt 2.  LOWRANK: [P | Q] gives P Q'; rank one gives the outer
    # product.  COMPLEMENT: 1 - A.  GRAM: P P' by hand.
    D = uo.factor_tensor(uo.DIST, np.zeros((3, 1)), 1, np.array([[0.0], [1.0], [3.0]]))
    assert np.array_equal(D, np.array([[0, 1, 3], [1, 0, 2], [3, 2, 0]], dtype=float))
    sq = uo.factor_tensor(uo.DIST, np.zeros((4, 1)), 2, np.array([[0.0, 0], [1, 0], [0, 1], [1, 1]]))
    assert sq[0, 1] == 1.0 and sq[0, 3] == pytest.approx(math.sqrt(2.0), rel=1e-15) and sq[2, 2] == 0.0
    u, v = np.array([1.0, 2.0, -1.0]), np.array([3.0, 0.5, 2.0])
    L = uo.factor_tensor(uo.LOWRANK, np.zeros((3, 1)), 1, np.stack([u, v], axis=1))
    assert np.array_equal(L, np.outer(u, v))
    P = np.arange(6.0).reshape(3, 2)
    Q = np.array([[1.0, -1.0], [0.5, 2.0], [0.0, 3.0]])
    L2 = uo.factor_tensor(uo.LOWRANK, np.zeros((3, 1)), 2, np.hstack([P, Q]))
    assert L2[2, 1] == P[2, 0] * Q[1, 0] + P[2, 1] * Q[1, 1]
    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    assert np.array_equal(uo.factor_tensor(uo.COMPLEMENT, np.zeros((2, 1)), 1, A), np.array([[1.0, 0], [0, 1]]))
    # GRAM: P P', the squared row norms on the diagonal; the first `param` columns only
    Gm = uo.factor_tensor(uo.GRAM, np.zeros((3, 1)), 2, P)
    assert np.array_equal(Gm, np.array([[1.0, 3, 5], [3, 13, 23], [5, 23, 41]]))
    assert np.array_equal(uo.factor_tensor(uo.GRAM, np.zeros((3, 1)), 1, P), np.outer(P[:, 0], P[:, 0]))
