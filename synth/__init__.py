"""Seeded synthetic inputs and workload descriptions.

This module is shared by the CUDA path's tests/benchmark and by the FP64 oracle.
It holds only input generation and the plain description of each workload (the
kernel graph, the factor kinds, the sizes and the seeds); it holds none of the
method's arithmetic (no kernel maps, no partitions, no contractions).

Workloads stand in for the paper's experiments (HOIF chains at n <= 1e4, motif
adjacency at n <= 2e4; Section 4) with the shapes named below.  All draws use
numpy's PCG64 ``default_rng``.

Graph convention: vertices 0..m-1; an edge ``(a, b, f)`` is the ordered pair
factor ``F_f(x_a, x_b)`` (the paper's multiplicative decomposition, Section 3.1,
with signature tuples of length 2); a unary ``(v, f)`` is ``f(x_v)`` (tuple of
length 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Factor kinds (same numbering as include/ustat.h).
RBF = 0        # exp(-||x - y||^2 / h)
LINEAR = 1     # (x . y) / h
TANH_DOT = 2   # tanh(x . w), unary
MATRIX = 3     # caller-supplied n x n matrix
VECTOR = 4     # caller-supplied length-n vector
DIST = 5       # ||y_i - y_j|| between the rows of a caller-supplied n x p matrix Y
LOWRANK = 6    # sum_k P(i, k) Q(j, k) from caller-supplied n x r matrices, data = [P | Q]
COMPLEMENT = 7  # 1 - A for a caller-supplied n x n matrix A
GRAM = 8       # sum_k P(i, k) P(j, k) from a caller-supplied n x r matrix P (symmetric)


@dataclass
class Factor:
    kind: int
    param: float = 1.0
    data: np.ndarray | None = None   # w for TANH_DOT, the matrix/vector for MATRIX/VECTOR


@dataclass
class Graph:
    m: int
    edges: list = field(default_factory=list)   # (a, b, factor_id)
    unary: list = field(default_factory=list)   # (v, factor_id)


def normal_X(n: int, d: int, seed: int) -> np.ndarray:
    """n x d iid N(0, 1), float64, row-major."""
    return np.random.default_rng(seed).standard_normal((n, d))


def student_t_X(n: int, d: int, seed: int, df: float = 5.0) -> np.ndarray:
    """n x d iid Student-t(df), rounded to float32 (the stored values are the sample)."""
    return np.random.default_rng(seed).standard_t(df, (n, d)).astype(np.float32)


def tanh_weight(d: int, seed: int = 1) -> np.ndarray:
    """w ~ N(0, I_d / d), float64."""
    return np.random.default_rng(seed).standard_normal(d) / np.sqrt(d)


def batched_sizes(count: int = 512, lo: int = 256, hi: int = 4096, seed: int = 0) -> np.ndarray:
    """Sample sizes n_i ~ uniform integers in [lo, hi] (inclusive)."""
    return np.random.default_rng(seed).integers(lo, hi + 1, count)


def cycle(m: int, factor: int = 0) -> Graph:
    return Graph(m, [(i, (i + 1) % m, factor) for i in range(m)], [])


def path(m: int, factor: int = 0) -> Graph:
    return Graph(m, [(i, i + 1, factor) for i in range(m - 1)], [])


def complete(m: int, factor: int = 0) -> Graph:
    return Graph(m, [(a, b, factor) for a in range(m) for b in range(a + 1, m)], [])


def triangle_graph() -> Graph:
    return cycle(3)


def cycle4_graph() -> Graph:
    return cycle(4)


def path5_chord_graph() -> Graph:
    """Path 1-2-3-4-5 plus chord 1-3, unary factor 1 on vertex 5 (0-based: 4)."""
    return Graph(5, [(0, 1, 0), (1, 2, 0), (2, 3, 0), (3, 4, 0), (0, 2, 0)], [(4, 1)])


def k4_plus_cycle_graph() -> Graph:
    """K4 on 1..4 plus edges 4-5, 5-6, 6-1 (0-based K4 on 0..3, then 3-4, 4-5, 5-0)."""
    g = complete(4)
    return Graph(6, g.edges + [(3, 4, 0), (4, 5, 0), (5, 0, 0)], [])


def rbf(d: int) -> Factor:
    return Factor(RBF, float(2 * d))


def linear(d: int) -> Factor:
    return Factor(LINEAR, float(d))


@dataclass
class Workload:
    name: str
    graph: Graph
    factors: list
    n: int
    d: int
    X: np.ndarray


def workload(name: str, n: int | None = None) -> Workload:
    """The five workloads, by name.  ``n`` overrides the sample size (same seed and
    distribution, first ``n`` draws are NOT reused: the whole sample is redrawn)."""
    if name == "triangle_rbf":
        n = 200 if n is None else n
        d = 8
        return Workload(name, triangle_graph(), [rbf(d)], n, d, normal_X(n, d, 0))
    if name == "c4_rbf":
        n = 4096 if n is None else n
        d = 32
        return Workload(name, cycle4_graph(), [rbf(d)], n, d, normal_X(n, d, 0))
    if name == "path5_chord_linear_tanh":
        n = 16384 if n is None else n
        d = 64
        w = tanh_weight(d, 1)
        return Workload(name, path5_chord_graph(), [linear(d), Factor(TANH_DOT, 1.0, w)], n, d,
                        student_t_X(n, d, 0))
    if name == "k4_cycle_rbf":
        n = 1024 if n is None else n
        d = 32
        return Workload(name, k4_plus_cycle_graph(), [rbf(d)], n, d, normal_X(n, d, 0))
    raise KeyError(name)


def batched_workload(count: int = 512, d: int = 16, lo: int = 256, hi: int = 4096):
    """Independent samples of uneven size: list of (n_i, X_i) with X_i ~ N(0,1),
    n_i from seed 0 and sample i from seed 1000 + i."""
    sizes = batched_sizes(count, lo, hi, 0)
    return [(int(n), normal_X(int(n), d, 1000 + i)) for i, n in enumerate(sizes)]


def ternary_vector(n: int, seed: int) -> np.ndarray:
    """Entries uniform in {-1, 0, 1}, float64 (integer-valued factor inputs)."""
    return np.random.default_rng(seed).integers(-1, 2, n).astype(np.float64)


def random_connected_graph(rng: np.random.Generator, m: int, p: float, max_unary: int = 2) -> Graph:
    """Connected G(m, p): edges kept with probability p, a random spanning tree
    added so the graph is connected; up to ``max_unary`` unary factors (id 1)."""
    keep = set()
    for a in range(m):
        for b in range(a + 1, m):
            if rng.random() < p:
                keep.add((a, b))
    perm = rng.permutation(m)
    for i in range(1, m):
        a, b = int(perm[i]), int(perm[rng.integers(0, i)])
        keep.add((min(a, b), max(a, b)))
    edges = [(a, b, 0) for (a, b) in sorted(keep)]
    nu = int(rng.integers(0, max_unary + 1))
    unary = [(int(v), 1) for v in rng.choice(m, nu, replace=False)]
    return Graph(m, edges, unary)


# --------------------------------------------------------------------------------------
# Motif counts (Section 4.2 and its appendix): an Erdos-Renyi adjacency matrix A and
# B = 1 - A; an induced motif r on k vertices is the U-statistic of the kernel that
# puts A on the motif's edges and B on every other pair, divided by |Aut(r)|.
# --------------------------------------------------------------------------------------

def er_adjacency(n: int, p: float, seed: int) -> np.ndarray:
    """Adjacency matrix of G(n, p): each of the n (n - 1) / 2 pairs is an edge
    independently with probability p (the pair i < j decided by the draw in row
    i, column j).  Symmetric, 0 / 1, float64, zero diagonal."""
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n), dtype=np.float64)
    cols = np.arange(n)
    for r0 in range(0, n, 1024):
        r1 = min(n, r0 + 1024)
        blk = rng.random((r1 - r0, n)) < p
        blk &= cols[None, :] > np.arange(r0, r1)[:, None]
        A[r0:r1] = blk
    A += A.T
    return A


# name: (k, edges of the motif on vertices 0..k-1).  The eleven graphs on four
# vertices and the four on three, up to isomorphism; the paper's r1..r8 are
# vshape, triangle, star3, path4, paw, cycle4, diamond, clique4.
MOTIFS = {
    "empty3": (3, []),
    "edge3": (3, [(0, 1)]),
    "vshape": (3, [(0, 1), (1, 2)]),
    "triangle": (3, [(0, 1), (1, 2), (0, 2)]),
    "empty4": (4, []),
    "edge4": (4, [(0, 1)]),
    "matching4": (4, [(0, 1), (2, 3)]),
    "vshape4": (4, [(0, 1), (1, 2)]),
    "triangle4": (4, [(0, 1), (1, 2), (0, 2)]),
    "star3": (4, [(0, 1), (0, 2), (0, 3)]),
    "path4": (4, [(0, 1), (1, 2), (2, 3)]),
    "paw": (4, [(0, 1), (0, 2), (1, 2), (2, 3)]),
    "cycle4": (4, [(0, 1), (1, 2), (2, 3), (0, 3)]),
    "diamond": (4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3)]),
    "clique4": (4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]),
}
CONNECTED4 = ["star3", "path4", "paw", "cycle4", "diamond", "clique4"]


def motif_graph(name: str):
    """The kernel graph of an induced motif: an edge (a, b) for every pair of the
    k vertices, with factor "A" on the motif's edges and "B" elsewhere.  Returns
    (Graph, the matrix name of each factor id)."""
    k, medges = MOTIFS[name]
    on = {frozenset(e) for e in medges}
    names = []
    edges = []
    for a in range(k):
        for b in range(a + 1, k):
            s = "A" if frozenset((a, b)) in on else "B"
            if s not in names:
                names.append(s)
            edges.append((a, b, names.index(s)))
    return Graph(k, edges), names


def motif_factors(names, A: np.ndarray, B: np.ndarray | None = None) -> list:
    """MATRIX factors for a motif graph's factor names; B = 1 - A unless given."""
    if "B" in names and B is None:
        B = 1.0 - A
    return [Factor(MATRIX, 1.0, A if s == "A" else B) for s in names]


# --------------------------------------------------------------------------------------
# Distance covariance (Section 4.3): a synthetic stand-in for monthly log-returns of the
# stocks of 11 sectors over n = 138 months.
# --------------------------------------------------------------------------------------

def sector_returns(n: int = 138, sectors: int = 11, seed: int = 0) -> list:
    """One n x p_k matrix per sector, p_k uniform in [20, 70]: a market factor
    (sd 0.04) and a sector factor (sd 0.03) with loadings uniform in [0.5, 1.5],
    plus Student-t(4) noise scaled by 0.05; float64."""
    rng = np.random.default_rng(seed)
    dims = rng.integers(20, 71, sectors)
    market = 0.04 * rng.standard_normal(n)
    out = []
    for k in range(sectors):
        s = 0.03 * rng.standard_normal(n)
        p = int(dims[k])
        beta = rng.uniform(0.5, 1.5, p)
        gamma = rng.uniform(0.5, 1.5, p)
        eps = 0.05 * rng.standard_t(4.0, (n, p))
        out.append(market[:, None] * beta[None, :] + s[:, None] * gamma[None, :] + eps)
    return out


# --------------------------------------------------------------------------------------
# Higher-order influence functions (Section 4.1): chain U-statistics of the pairwise
# factors g(X_1, X_2) = A_1 phi(Z_1)' A_2 phi(Z_2) and f(X_1, X_2) = A_1 phi(Z_1)' phi(Z_2) Y_2.
# --------------------------------------------------------------------------------------

def hoif_sample(n: int, k: int = 16, seed: int = 0):
    """An unconfounded observational sample with a k-dimensional dictionary:
    Z ~ N(0, I_k), treatment A ~ Bernoulli(1/2) independent of Z, outcome
    Y = Z . beta + N(0, 1) with beta ~ N(0, I_k / k), and phi(Z) = sqrt(2) Z, so
    that the mean of A phi(Z) phi(Z)' is the identity (the paper's simplifying
    assumption).  Returns (phi, A, Y): n x k, n, n, float64."""
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((n, k))
    A = (rng.random(n) < 0.5).astype(np.float64)
    beta = rng.standard_normal(k) / np.sqrt(k)
    Y = Z @ beta + rng.standard_normal(n)
    return np.sqrt(2.0) * Z, A, Y


def hoif_chain_graph(j: int) -> Graph:
    """The kernel graph of h_j (the paper's equation for the HOIF kernel): the
    chain 0 - 1 - ... - (j-1), factor 0 = g on its first j - 2 edges and factor
    1 = f on the last one (for j = 2 only f, as factor id 0)."""
    if j == 2:
        return Graph(2, [(0, 1, 0)])
    return Graph(j, [(v, v + 1, 0) for v in range(j - 2)] + [(j - 2, j - 1, 1)])
