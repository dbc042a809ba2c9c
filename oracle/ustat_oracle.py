"""FP64 CPU oracle: exact U-statistics by the partition sum of restricted V-statistics.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import this module.  It shares no code with the
CUDA path (paper_2508_12627_gb300/) and never imports it.

Everything here restates the paper's definitions (arXiv 2508.12627) in float64:

* U-statistic as the sum over ordered distinct m-tuples (Section 2.1, Definition
  "U-Statistic"); V-statistic over all of [n]^m (Definition "V-Statistic").
* Multiplicative decomposition h = prod_k h_k(x[A_k]) and tensorization
  T_k(alpha) = h_k(X[alpha]) (Section 3.1, Definition "Multiplicative
  Decomposition", Algorithm 1).
* Partitions of [m] (Section 2.3, Definition "Partition"), enumerated as
  restricted growth strings in lexicographic order.
* Moebius coefficients mu_pi = (-1)^(m-|pi|) prod_C (|C|-1)! (Section 3.3, Lemma
  "Decomposition of U-Statistic into V-Statistics") and, independently, the
  Moebius function of the partition lattice from its defining recursion
  (Appendix E, Definition "Moebius Function").
* The restricted V-statistic V_pi: the V-statistic of the kernel with the indices
  of each block of pi equal (Section 3.3, Definition "Restricted V-Statistic"),
  written as the Einsum of the quotient signature (the identity right after
  Example "A_pi").
* Einsum evaluated by summing out one index at a time along an elimination order
  (Section 3.2, Proposition "complexity_einsum" and its proof in Appendix D);
  a matrix product is used as a library primitive for the sum over v of
  (vector on v) x (matrices on (v,w), (v,x)) and, with the (w, x) pairs as rows,
  x (matrix on (v,y)).
* Sparsified tensors T~ (Lemma "sparsification_trick") and the surviving set
  Pi_m^A (Remark after it, equation "quotient_set").
* U = sum_pi mu_pi V_pi over all partitions (Section 3.3, Lemma "Decomposition of
  U-Statistic into V-Statistics").

Readings where the paper is silent (kept identical on both sides of the test):
* the RBF kernel is exp(-||x-y||^2 / h) with h = 2d; the linear kernel x.y / h with
  h = d; the unary factor is tanh(x . w);
* an intra-block pairwise factor F(x_a, x_b) with a, b in one block contributes
  F(x_i, x_i), the diagonal, exactly as Definition "Restricted V-Statistic" gives.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

# Factor kinds (plain integers; the same numbering is used by the input module).
RBF, LINEAR, TANH_DOT, MATRIX, VECTOR, DIST, LOWRANK, COMPLEMENT, GRAM = 0, 1, 2, 3, 4, 5, 6, 7, 8


# --------------------------------------------------------------------------------------
# Partitions and Moebius coefficients (Section 2.3; Section 3.3; Appendix E)
# --------------------------------------------------------------------------------------

def set_partitions(m: int) -> list[tuple[int, ...]]:
    """All partitions of [m] as restricted growth strings a (a[0] = 0,
    a[i] <= 1 + max(a[:i])), in lexicographic order.  Block j of the partition is
    {i : a[i] == j}."""
    out = []

    def rec(prefix, top):
        if len(prefix) == m:
            out.append(tuple(prefix))
            return
        for b in range(top + 2):
            rec(prefix + [b], max(top, b))

    if m == 0:
        return [()]
    rec([0], 0)
    return out


def blocks(rgs) -> list[list[int]]:
    k = max(rgs) + 1 if rgs else 0
    return [[i for i, b in enumerate(rgs) if b == j] for j in range(k)]


def mu_closed_form(rgs) -> int:
    """mu_pi = (-1)^(m - |pi|) prod_{C in pi} (|C| - 1)!  (Lemma, Section 3.3)."""
    bl = blocks(rgs)
    sign = -1 if (len(rgs) - len(bl)) % 2 else 1
    return sign * math.prod(math.factorial(len(c) - 1) for c in bl)


def refines(pi, rho) -> bool:
    """pi <= rho in the refinement order: every block of pi lies inside a block of rho
    (Appendix E, Definition "Refinement of Partitions")."""
    for c in blocks(pi):
        if len({rho[i] for i in c}) != 1:
            return False
    return True


def mobius_lattice(m: int) -> dict:
    """mu(pi, rho) for all pi <= rho in the partition lattice of [m], from the
    defining recursion mu(s,s) = 1, mu(s,u) = -sum_{s <= t < u} mu(s,t)
    (Appendix E, Definition "Moebius Function").  Brute force; small m only."""
    parts = set_partitions(m)
    # number of blocks is a grading: t < u implies |t| > |u|
    order = sorted(parts, key=lambda p: -(max(p) + 1))
    mu = {}
    for s in parts:
        above = [u for u in order if refines(s, u)]
        for u in above:
            if u == s:
                mu[(s, u)] = 1
                continue
            acc = 0
            for t in above:
                if t != u and refines(t, u) and (s, t) in mu:
                    acc += mu[(s, t)]
            mu[(s, u)] = -acc
    return mu


def falling_factorial(n: int, m: int) -> int:
    """(n)_m = n (n-1) ... (n-m+1): the number of ordered distinct m-tuples of [n]."""
    return math.prod(range(n - m + 1, n + 1)) if m > 0 else 1


# --------------------------------------------------------------------------------------
# Tensorization (Section 3.1, Algorithm 1)
# --------------------------------------------------------------------------------------

def factor_tensor(kind: int, X: np.ndarray, param: float = 1.0, data=None) -> np.ndarray:
    """T_k(alpha) = h_k(X[alpha]) for one factor, in float64.

    RBF:      T(i, j) = exp(-||x_i - x_j||^2 / param), computed from the differences.
    LINEAR:   T(i, j) = (x_i . x_j) / param.
    TANH_DOT: T(i)    = tanh(x_i . w), w = data.
    MATRIX / VECTOR: the given data (float64).
    DIST:     T(i, j) = ||y_i - y_j|| for the rows of Y = data (the distance
              matrices of dCov, Section 4.3).
    LOWRANK:  T(i, j) = sum_k P(i, k) Q(j, k), data = [P | Q] with param = the
              number of columns of P (the HOIF factors, Section 4.1).
    COMPLEMENT: T = 1 - A, A = data (the motif kernels' non-edge factor,
              Section 4.2).
    GRAM:     T(i, j) = sum_k P(i, k) P(j, k), data = P with param = its number of
              columns (the symmetric HOIF factor g, Section 4.1)."""
    X = np.asarray(X, dtype=np.float64)
    if kind == RBF:
        diff = X[:, None, :] - X[None, :, :]
        return np.exp(-np.einsum("ijk,ijk->ij", diff, diff) / param)
    if kind == LINEAR:
        return (X @ X.T) / param
    if kind == TANH_DOT:
        return np.tanh(X @ np.asarray(data, dtype=np.float64))
    if kind in (MATRIX, VECTOR):
        return np.asarray(data, dtype=np.float64)
    if kind == DIST:
        Y = np.asarray(data, dtype=np.float64)
        Y = Y.reshape(Y.shape[0], -1)
        diff = Y[:, None, :] - Y[None, :, :]
        return np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))
    if kind == LOWRANK:
        D = np.asarray(data, dtype=np.float64)
        r = int(param)
        return D[:, :r] @ D[:, r:2 * r].T
    if kind == COMPLEMENT:
        return 1.0 - np.asarray(data, dtype=np.float64)
    if kind == GRAM:
        D = np.asarray(data, dtype=np.float64)
        return D[:, :int(param)] @ D[:, :int(param)].T
    raise ValueError(kind)


def factor_arity(kind: int) -> int:
    return 1 if kind in (TANH_DOT, VECTOR) else 2


def signature(graph) -> list[tuple[tuple[int, ...], int]]:
    """The decomposition signature A = (A_k) with each tuple's factor id:
    edges give (a, b), unary factors give (v,)."""
    sig = [((a, b), f) for (a, b, f) in graph.edges]
    sig += [((v,), f) for (v, f) in graph.unary]
    return sig


def tensorize(graph, factors, X) -> dict:
    """Algorithm 1: one tensor per factor id (each factor is tensorized once even if
    it appears in several signature tuples)."""
    used = sorted({f for _, f in signature(graph)})
    out = {}
    for f in used:
        fa = factors[f]
        out[f] = factor_tensor(fa.kind, X, fa.param, fa.data)
    return out


def sparsify(T: np.ndarray) -> np.ndarray:
    """T~ of Lemma "sparsification_trick": zero every entry whose index tuple repeats
    an index (the diagonal of a matrix); a vector is unchanged."""
    if T.ndim == 2:
        T = T.copy()
        np.fill_diagonal(T, 0.0)
    return T


def survives(sig, rgs) -> bool:
    """pi in Pi_m^A (equation "quotient_set"): no block holds two indices of one tuple."""
    for tup, _ in sig:
        labels = [rgs[i] for i in tup]
        if len(set(labels)) < len(labels):
            return False
    return True


# --------------------------------------------------------------------------------------
# The quotient signature (each index replaced by its block; Section 3.3, the induced
# notation of Example "A_pi") and the Einsum by one-index-at-a-time elimination
# (Section 3.2, Proposition "complexity_einsum", Appendix D)
# --------------------------------------------------------------------------------------

def induced_notation(sig, rgs):
    """The signature with every index replaced by the label of its block."""
    return [(tuple(rgs[i] for i in tup), f) for tup, f in sig]


def _canonical(axes, arr):
    """Express a factor on distinct, sorted axes.  A repeated axis (j, j) reads the
    diagonal T(i, i), which is what Definition "Einsum Operation" gives for a tuple
    with a repeated index."""
    axes = list(axes)
    arr = np.asarray(arr)
    while len(set(axes)) < len(axes):
        # find the first repeated pair and take the diagonal over it
        for p in range(len(axes)):
            q = next((q for q in range(p + 1, len(axes)) if axes[q] == axes[p]), None)
            if q is not None:
                arr = np.diagonal(arr, axis1=p, axis2=q)  # diagonal axis goes last
                ax = axes[p]
                axes = [a for t, a in enumerate(axes) if t not in (p, q)] + [ax]
                break
    perm = sorted(range(len(axes)), key=lambda t: axes[t])
    return tuple(axes[t] for t in perm), np.transpose(arr, perm)


def min_degree_order(n_vertices, tensors):
    """An elimination order: repeatedly take the vertex with the fewest neighbours in
    the current interaction graph (ties: lowest label).  Any order gives the same
    exact value; this one only keeps intermediates small."""
    adj = {v: set() for v in range(n_vertices)}
    for axes, _ in tensors:
        for a in axes:
            adj[a].update(b for b in axes if b != a)
    alive = set(range(n_vertices))
    order = []
    while alive:
        v = min(alive, key=lambda u: (len(adj[u] & alive), u))
        nb = adj[v] & alive
        for a in nb:
            adj[a].update(nb - {a})
        alive.remove(v)
        order.append(v)
    return order


def einsum_eliminate(n_vertices, tensors, order=None, trace=None) -> float:
    """Einsum(T, A) with empty output: sum out one index at a time.

    ``tensors`` is a list of (axes, array).  Step for index v: multiply every
    tensor that carries v and sum over v; the product is a new tensor on the other
    indices it carried.  The product-and-sum of a vector on v with two or three
    matrices on (v, w), (v, x) [, (v, y)] is done by a matrix product; anything
    else by numpy.einsum.

    With ``trace`` (a list), each step appends the sorted index tuples of the
    tensors left after it, () standing for a scalar it produced: the Einsum
    notation sequence A_1, ..., A_m of Appendix D (Definition "Einsum Notation
    Sequence")."""
    work = [_canonical(ax, a) for ax, a in tensors]
    if order is None:
        order = min_degree_order(n_vertices, work)
    scalar = 1.0
    for v in order:
        group = [(ax, a) for ax, a in work if v in ax]
        work = [(ax, a) for ax, a in work if v not in ax]
        if not group:
            # an index no factor touches still ranges over [n]; there is none here
            # because every vertex belongs to the index set (Definition "Einsum
            # Notation") -- but a block with only intra-block factors collapses to
            # vectors, which do carry v.
            raise ValueError("index %d appears in no factor" % v)
        ax_out, arr = _sum_out(v, group)
        if ax_out:
            work.append((ax_out, arr))
        else:
            scalar *= float(arr)
        if trace is not None:
            trace.append(sorted(ax for ax, _ in work) + ([] if ax_out else [()]))
    for ax, a in work:   # only 0-d tensors can remain
        assert not ax
        scalar *= float(a)
    return scalar


def _sum_out(v, group):
    # Hadamard-merge tensors on the same axis set first.
    merged = {}
    for ax, a in group:
        merged[ax] = merged[ax] * a if ax in merged else a.copy()
    vec = merged.pop((v,), None)
    others = sorted({b for ax in merged for b in ax if b != v})
    mats = {ax: a for ax, a in merged.items() if len(ax) == 2}
    if len(mats) == len(merged) and len(others) <= 3 and all(len(ax) == 2 for ax in merged):
        # vector and matrices on (v, w): orient every matrix as M[v_index, w_index]
        oriented = []
        for ax, a in mats.items():
            w = ax[0] if ax[1] == v else ax[1]
            oriented.append((w, a if ax[0] == v else a.T))
        u = vec if vec is not None else None
        if len(oriented) == 0:
            return (), np.sum(u)
        if len(oriented) == 1:
            w, M = oriented[0]
            r = (u @ M) if u is not None else M.sum(axis=0)
            return (w,), r
        if len(oriented) == 2 and oriented[0][0] != oriented[1][0]:
            (w, A), (x, B) = sorted(oriented, key=lambda t: t[0])
            Bs = B * u[:, None] if u is not None else B
            return (w, x), A.T @ Bs
        if len(oriented) == 3:
            # three neighbours: T(w, x, y) = sum_v u(v) A(v, w) B(v, x) C(v, y), the
            # same sum with the (w, x) pairs laid out as the rows of one matrix
            (w, A), (x, B), (y, C) = sorted(oriented, key=lambda t: t[0])
            P = A[:, :, None] * B[:, None, :]
            if u is not None:
                P *= u[:, None, None]
            T = P.reshape(P.shape[0], -1).T @ C
            return (w, x, y), T.reshape(A.shape[1], B.shape[1], C.shape[1])
    # generic: numpy.einsum over the group
    letters = {}
    for ax in list(merged) + ([(v,)] if vec is not None else []):
        for b in ax:
            letters.setdefault(b, chr(ord("a") + len(letters)))
    ops, subs = [], []
    for ax, a in merged.items():
        ops.append(a)
        subs.append("".join(letters[b] for b in ax))
    if vec is not None:
        ops.append(vec)
        subs.append(letters[v])
    out_axes = tuple(b for b in sorted(letters) if b != v)
    spec = ",".join(subs) + "->" + "".join(letters[b] for b in out_axes)
    return out_axes, np.einsum(spec, *ops)


# --------------------------------------------------------------------------------------
# V_pi and U (Section 3.3, Definition "Restricted V-Statistic" and Lemma
# "Decomposition of U-Statistic into V-Statistics")
# --------------------------------------------------------------------------------------

def v_pi(sig, tensors, rgs) -> float:
    """V_pi = Einsum(T, A_pi) (Section 3.3): the restricted V-statistic of Definition
    "Restricted V-Statistic", evaluated on the induced notation."""
    ind = induced_notation(sig, rgs)
    k = max(rgs) + 1
    return einsum_eliminate(k, [(tup, tensors[f]) for tup, f in ind])


def ustat(graph, factors, X, sparse: bool = False, partitions=None, absolute: bool = False):
    """U = sum_pi mu_pi V_pi (Lemma "Decomposition of U-Statistic into
    V-Statistics"), returning a dict with
    ``U_sum`` (the paper's unnormalised sum over ordered distinct tuples),
    ``U_mean`` = U_sum / (n)_m, and per-partition ``rgs``, ``mu`` and ``V``.

    With ``sparse`` the tensors are T~ and only partitions in Pi_m^A are evaluated
    (the others are reported as V = 0); otherwise V_pi of the original tensors is
    computed for every partition.  With ``absolute`` every tensor is replaced by
    its entrywise absolute value: V_pi is then the sum of |terms| of V_pi, the
    scale against which rounding errors of a sum with cancellation are judged."""
    X = np.asarray(X)
    n = X.shape[0]
    m = graph.m
    sig = signature(graph)
    T = tensorize(graph, factors, X)
    if absolute:
        T = {f: np.abs(a) for f, a in T.items()}
    if sparse:
        T = {f: sparsify(a) for f, a in T.items()}
    parts = set_partitions(m) if partitions is None else partitions
    V, MU = [], []
    for rgs in parts:
        MU.append(mu_closed_form(rgs))
        if sparse and not survives(sig, rgs):
            V.append(0.0)
        else:
            V.append(v_pi(sig, T, rgs))
    u_sum = math.fsum(mu * v for mu, v in zip(MU, V))
    ff = falling_factorial(n, m)
    return {"U_sum": u_sum, "U_mean": u_sum / ff if ff else float("nan"),
            "rgs": parts, "mu": MU, "V": V}


# --------------------------------------------------------------------------------------
# Treewidth by definition (Section 2.3, Definitions "Vertex Elimination", "Treewidth")
# --------------------------------------------------------------------------------------

def treewidth_bruteforce(k: int, edges) -> int:
    """min over all elimination orders of the max degree at elimination.  k! orders;
    small graphs only."""
    if k == 0:
        return 0
    base = {v: set() for v in range(k)}
    for a, b in edges:
        if a != b:
            base[a].add(b)
            base[b].add(a)
    best = k
    for order in itertools.permutations(range(k)):
        adj = {v: set(s) for v, s in base.items()}
        worst = 0
        for v in order:
            nb = adj[v]
            worst = max(worst, len(nb))
            if worst >= best:
                break
            for a in nb:
                adj[a] |= nb - {a}
                adj[a].discard(v)
            del adj[v]
        best = min(best, worst)
    return best


def quotient_edges(graph, rgs):
    """Edges of the quotient graph G/pi (Section 2.3, Definition "Quotient Graph")."""
    es = set()
    for a, b, _ in graph.edges:
        p, q = rgs[a], rgs[b]
        if p != q:
            es.add((min(p, q), max(p, q)))
    return sorted(es)
