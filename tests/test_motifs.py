"""Motif counts as U-statistics (Section 4.2, Appendix I): an induced motif r on
k vertices is the U-statistic of the kernel with A on r's edges and B = 1 - A on
the other pairs, divided by |Aut(r)|.

CPU: the motif kernel graphs and |Aut| against the paper's constants; the
oracle's counts against brute-force enumeration of vertex subsets; closed forms
on complete and empty graphs; and the subgraph-count identities that the
full-size GPU checks use, against brute force.  GPU: every 3- and 4-vertex type
bit-exact against the oracle at n = 130 (two tiles and a ragged tail) in every
precision, and the censuses at the paper's sizes (all 3-vertex types at
n = 20000, all 4-vertex types at n = 2000) through integrality and the
identities."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import ustat_oracle as uo
from tests.conftest import GOLDEN

NAMES3 = [k for k, (m, _) in synth.MOTIFS.items() if m == 3]
NAMES4 = [k for k, (m, _) in synth.MOTIFS.items() if m == 4]


def _aut(k, edges):
    E = {frozenset(e) for e in edges}
    return sum(1 for p in itertools.permutations(range(k)) if {frozenset((p[a], p[b])) for a, b in edges} == E)


def _canon(k, edges):
    # least sorted edge list over all relabellings: equal iff isomorphic
    return min(tuple(sorted(tuple(sorted((p[a], p[b]))) for a, b in edges)) for p in itertools.permutations(range(k)))


CANON = {name: _canon(k, e) for name, (k, e) in synth.MOTIFS.items()}


def brute_census(A, k):
    """Number of k-subsets of vertices whose induced subgraph is of each type."""
    n = A.shape[0]
    names = NAMES3 if k == 3 else NAMES4
    by = {CANON[nm]: nm for nm in names}
    out = dict.fromkeys(names, 0)
    for S in itertools.combinations(range(n), k):
        e = [(i, j) for i in range(k) for j in range(i + 1, k) if A[S[i], S[j]]]
        out[by[_canon(k, e)]] += 1
    return out


def oracle_count(name, A):
    g, fn = synth.motif_graph(name)
    r = uo.ustat(g, synth.motif_factors(fn, A), np.zeros((A.shape[0], 1)))
    return r["U_sum"], r


# patterns whose (not necessarily induced) copies in G have closed forms
PATTERNS = {
    "edge": (2, [(0, 1)]),
    "p2": (3, [(0, 1), (1, 2)]),
    "k3": (3, [(0, 1), (1, 2), (0, 2)]),
    "s3": (4, [(0, 1), (0, 2), (0, 3)]),
    "m2": (4, [(0, 1), (2, 3)]),
    "p3": (4, [(0, 1), (1, 2), (2, 3)]),
    "c4": (4, [(0, 1), (1, 2), (2, 3), (0, 3)]),
    "k4": (4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]),
}


def copies_in(k, edges, pattern):
    """Copies of a pattern (subgraphs, not necessarily induced) in a graph on k vertices."""
    kp, pe = pattern
    if kp > k:
        return 0
    E = {frozenset(e) for e in edges}
    maps = sum(1 for f in itertools.permutations(range(k), kp) if all(frozenset((f[a], f[b])) in E for a, b in pe))
    return maps // _aut(kp, pe)


def triangles_by_neighbourhoods(A):
    """Triangles: for each vertex, the edges among its neighbours (each triangle
    is seen from its three vertices)."""
    s = 0
    for u in range(A.shape[0]):
        N = np.flatnonzero(A[u])
        s += int(A[np.ix_(N, N)].sum()) // 2
    return s // 3


def pattern_totals(A, with4=True):
    """Copies of each pattern in G from closed forms in the degrees, A^2 and the
    neighbourhoods (exact integers)."""
    d = A.sum(1).astype(np.int64)
    E = int(d.sum()) // 2
    T = triangles_by_neighbourhoods(A)
    P2 = int((d * (d - 1) // 2).sum())
    out = {"edge": E, "p2": P2, "k3": T}
    if not with4:
        return out
    out["s3"] = int((d * (d - 1) * (d - 2) // 6).sum())
    out["m2"] = E * (E - 1) // 2 - P2
    iu, ju = np.nonzero(np.triu(A, 1))
    out["p3"] = int(((d[iu] - 1) * (d[ju] - 1)).sum()) - 3 * T
    A2 = A @ A                              # float64, exact for these integers
    # closed 4-walks: 8 per 4-cycle, 4 per 2-path, 2 per edge
    out["c4"] = (int(round(float((A2 * A2).sum()))) - 4 * P2 - 2 * E) // 8
    # 4-cliques: for each edge, the edges among the common neighbours (6 per clique)
    k4 = 0
    for u in range(A.shape[0]):
        N = np.flatnonzero(A[u])
        N = N[N > u]
        for v in N:
            C = np.flatnonzero(A[u] * A[v])
            k4 += int(A[np.ix_(C, C)].sum()) // 2
    out["k4"] = k4 // 6
    return out


def census_identities(counts, A, k):
    """Every pattern total equals the sum over induced types of (copies of the
    pattern in the type) x (count of the type); and the counts add up to C(n, k)."""
    n = A.shape[0]
    names = NAMES3 if k == 3 else NAMES4
    assert sum(counts[nm] for nm in names) == math.comb(n, k)
    tot = pattern_totals(A, with4=(k == 4))
    for pat, want in tot.items():
        kp = PATTERNS[pat][0]
        got = sum(copies_in(*synth.MOTIFS[nm], PATTERNS[pat]) * counts[nm] for nm in names)
        assert got == want * math.comb(n - kp, k - kp), (pat, got, want)


# ---------------------------------------------------------------- CPU


def test_motif_graphs_match_the_paper():
    gold = json.load(open(os.path.join(GOLDEN, "motif_automorphisms.json")))["motifs"]
    for r in gold.values():
        k, e = synth.MOTIFS[r["name"]]
        assert _aut(k, e) == r["aut"], r
    # the fifteen names are the graphs on 3 and 4 vertices, each once
    assert len({CANON[n] for n in NAMES3}) == 4 and len({CANON[n] for n in NAMES4}) == 11
    for name in synth.MOTIFS:
        g, fn = synth.motif_graph(name)
        k, e = synth.MOTIFS[name]
        assert sorted((a, b) for a, b, _ in g.edges) == [(a, b) for a in range(k) for b in range(a + 1, k)]
        on = {frozenset(x) for x in e}
        assert all((fn[f] == "A") == (frozenset((a, b)) in on) for a, b, f in g.edges)


def test_binding_builds_the_same_kernel_graphs():
    pytest.importorskip("torch")
    from paper_2508_12627_gb300 import motifs
    for name, (k, e) in synth.MOTIFS.items():
        g, fn = motifs.kernel_graph(k, e)
        gs, fs = synth.motif_graph(name)
        assert g.edges == gs.edges and fn == fs and g.m == gs.m
        assert motifs.automorphisms(k, e) == _aut(k, e)


@pytest.mark.parametrize("p,seed", [(0.3, 0), (0.6, 1)])
def test_oracle_counts_induced_subgraphs(p, seed):
    A = synth.er_adjacency(9, p, seed)
    for k in (3, 4):
        brute = brute_census(A, k)
        for name, want in brute.items():
            u, _ = oracle_count(name, A)
            aut = _aut(*synth.MOTIFS[name])
            assert u == want * aut, (name, u, want)


def test_complete_and_empty_graphs():
    n = 10
    full = np.ones((n, n)) - np.eye(n)
    for name in synth.MOTIFS:
        k = synth.MOTIFS[name][0]
        aut = _aut(*synth.MOTIFS[name])
        assert oracle_count(name, full)[0] == (math.perm(n, k) if name in ("triangle", "clique4") else 0)
        assert oracle_count(name, np.zeros((n, n)))[0] == (math.perm(n, k) if name in ("empty3", "empty4") else 0)
        assert math.perm(n, k) % aut == 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pattern_totals_and_census_identities_against_brute_force(seed):
    A = synth.er_adjacency(10, 0.5, seed)
    tot = pattern_totals(A)
    n = A.shape[0]
    for pat, (kp, pe) in PATTERNS.items():
        # brute force over injective maps of the pattern into G
        maps = sum(1 for f in itertools.permutations(range(n), kp) if all(A[f[a], f[b]] for a, b in pe))
        assert tot[pat] == maps // _aut(kp, pe), pat
    for k in (3, 4):
        census_identities(brute_census(A, k), A, k)


# ---------------------------------------------------------------- GPU


def _gpu_counts(A, names, precision):
    from paper_2508_12627_gb300 import build
    build.build()
    import torch
    from paper_2508_12627_gb300 import motifs
    mc = motifs.MotifCounter(A, precision=precision)
    out = {}
    for nm in names:
        k, e = synth.MOTIFS[nm]
        p, _, aut = mc.plan(k, e)
        o = torch.empty(2 + p.info["n_parts"], dtype=torch.float64, device="cuda")
        mc.ws.fill_(255)                                 # NaN bytes: no stale reads
        mc.launch(k, e, o)
        out[nm] = (o.cpu().numpy(), aut)
    return out


@pytest.fixture(scope="module")
def small_case():
    A = synth.er_adjacency(130, 0.3, 3)
    return A, {nm: oracle_count(nm, A)[1] for nm in synth.MOTIFS}


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["bf16x3", "bf16x4", "tf32", "fp32", "fp64"])
def test_every_motif_bit_exact_against_oracle(small_case, precision):
    A, ref = small_case
    got = _gpu_counts(A, list(synth.MOTIFS), precision)
    for nm, (o, aut) in got.items():
        assert o[0] == ref[nm]["U_sum"], (nm, o[0], ref[nm]["U_sum"])
        assert np.array_equal(o[2:], np.asarray(ref[nm]["V"])), nm
        assert o[0] % aut == 0


@pytest.mark.gpu
def test_three_vertex_census_at_n_20000():
    # the size of the paper's 3-vertex table; four unknowns, four exact equations
    A = synth.er_adjacency(20000, 0.005, 5)
    got = _gpu_counts(A, NAMES3, "bf16x3")
    counts = {}
    for nm, (o, aut) in got.items():
        assert o[0] % aut == 0 and o[0] < 2.0 ** 53
        counts[nm] = int(o[0]) // aut
    census_identities(counts, A, 3)


@pytest.mark.gpu
def test_four_vertex_census_at_n_2000():
    # the size of the paper's 4-vertex table; eleven types, nine exact equations
    A = synth.er_adjacency(2000, 0.1, 6)
    got = _gpu_counts(A, NAMES4, "bf16x3")
    counts = {}
    for nm, (o, aut) in got.items():
        assert o[0] % aut == 0 and o[0] < 2.0 ** 53
        counts[nm] = int(o[0]) // aut
    census_identities(counts, A, 4)


def test_planted_mistakes_fail_the_pins():
    # a wrong automorphism count or a swapped A / B edge breaks the brute-force pin
    A = synth.er_adjacency(9, 0.5, 7)
    brute = brute_census(A, 4)
    k, e = synth.MOTIFS["paw"]
    u, _ = oracle_count("paw", A)
    assert u == brute["paw"] * _aut(k, e)
    assert u != brute["paw"] * (_aut(k, e) * 2)               # |Aut| of the paw taken as 4
    g, fn = synth.motif_graph("paw")
    swapped = synth.Graph(g.m, [(a, b, 1 - f) if (a, b) == (2, 3) else (a, b, f) for a, b, f in g.edges])
    r = uo.ustat(swapped, synth.motif_factors(fn, A), np.zeros((9, 1)))
    assert r["U_sum"] != u                                      # the tail edge read from B instead of A


def test_five_vertex_clique_exceeds_the_engines_treewidth():
    # K5 needs a step with four neighbours: the planner refuses it before any device work
    pytest.importorskip("torch")
    from paper_2508_12627_gb300 import build
    build.build()
    from paper_2508_12627_gb300 import motifs, ustat as us
    edges = [(a, b) for a in range(5) for b in range(a + 1, 5)]
    g, names = motifs.kernel_graph(5, edges)
    with pytest.raises(us.UstatError) as e:
        us.Plan(g, [us.MATRIX] * len(names))
    assert e.value.code == us.USTAT_ERR_TW_TOO_LARGE
    # every induced 5-vertex motif carries A or B on all ten pairs, so its kernel
    # graph is K5 whatever the motif: the induced 5-cycle is refused as well
    g, names = motifs.kernel_graph(5, [(0, 1), (1, 2), (2, 3), (3, 4), (0, 4)])
    with pytest.raises(us.UstatError):
        us.Plan(g, [us.MATRIX] * len(names))
