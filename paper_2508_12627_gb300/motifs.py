"""Induced motif counts of a graph through the engine (the motif example of
Section 4.2 and Appendix I): a motif r on k vertices is counted by the
U-statistic of the kernel that puts the adjacency matrix A on r's edges and
B = 1 - A on every other pair of the k vertices, divided by |Aut(r)|:

    C(r, G) = (1 / |Aut(r)|) * sum over ordered distinct k-tuples of
              prod_{(a, b) in E(r)} A[i_a, i_b] * prod_{(a, b) not in E(r)} B[i_a, i_b]

    mc = MotifCounter(A, precision="bf16x3")          # A: n x n 0 / 1, symmetric
    mc.count(3, [(0, 1), (1, 2), (0, 2)])             # triangles

For 0 / 1 matrices every product entry, contraction and reduction of the
split-BF16 path is an integer held exactly (digits of 0 and 1 are exact, the
tensor-core accumulators sum at most n < 2^24 unit products, the reductions are
float64), so the counts are exact integers below 2^53.  A is uploaded once; B
enters as a COMPLEMENT factor of A, which the library forms on the device; the
sample argument of ustat_eval is a dummy n x 1 column, which these factors do
not read.  A caller-given B (other than 1 - A) is uploaded as a MATRIX factor.
"""
from __future__ import annotations

import itertools

import numpy as np
import torch

from . import ustat as us


class KernelGraph:
    def __init__(self, m, edges):
        self.m = m
        self.edges = edges
        self.unary = []


def kernel_graph(k, edges):
    """The kernel graph of motif (k, edges): one pairwise factor per pair of the
    k vertices, "A" on the motif's edges and "B" on the others.  Returns the
    graph and the matrix name of each factor id."""
    on = {frozenset(e) for e in edges}
    names, out = [], []
    for a in range(k):
        for b in range(a + 1, k):
            s = "A" if frozenset((a, b)) in on else "B"
            if s not in names:
                names.append(s)
            out.append((a, b, names.index(s)))
    return KernelGraph(k, out), names


def automorphisms(k, edges):
    """|Aut(r)|: the vertex permutations that map the edge set onto itself."""
    E = {frozenset(e) for e in edges}
    return sum(1 for p in itertools.permutations(range(k))
               if {frozenset((p[a], p[b])) for a, b in edges} == E)


class MotifCounter:
    """The device copy of A (and of B only when the caller gives one), one plan per
    motif (cached), one shared workspace."""

    def __init__(self, A, precision="bf16x3", device="cuda:0"):
        self.device = torch.device(device)
        A = np.ascontiguousarray(A, dtype=np.float64)
        self.n = A.shape[0]
        if A.shape != (self.n, self.n):
            raise ValueError("A must be n x n")
        self.precision = precision
        self.A = torch.empty((self.n, self.n), dtype=torch.float64, device=self.device)
        self.B = None   # a caller-given B; None: B = 1 - A, formed on the device
        self.X = torch.zeros((self.n, 1), dtype=torch.float64, device=self.device)
        self.plans = {}
        self.ws = None
        self.set_graph(A)

    def set_graph(self, A, B=None, non_blocking=False):
        """New adjacency matrix (numpy or a pinned host tensor); B = 1 - A (formed
        on the device) unless given."""
        src = A if isinstance(A, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(A, dtype=np.float64))
        self.A.copy_(src, non_blocking=non_blocking)
        if B is None:
            self.B = None
        else:
            if self.B is None:
                self.B = torch.empty_like(self.A)
            srcb = B if isinstance(B, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(B, dtype=np.float64))
            self.B.copy_(srcb, non_blocking=non_blocking)

    def plan(self, k, edges):
        key = (k, tuple(sorted(tuple(sorted(e)) for e in edges)), self.B is not None)
        if key not in self.plans:
            g, names = kernel_graph(k, edges)
            kinds = [us.MATRIX if s == "A" or self.B is not None else us.COMPLEMENT for s in names]
            p = us.Plan(g, kinds, precision=self.precision)
            need = max(256, p.workspace_bytes(self.n, 1))
            if self.ws is None or self.ws.numel() < need:
                self.ws = torch.empty(need, dtype=torch.uint8, device=self.device)
            self.plans[key] = (p, names, automorphisms(k, edges))
        return self.plans[key]

    def launch(self, k, edges, out, stream=None):
        """Enqueue one count; ``out`` is a float64 device tensor of 2 + Bell(k):
        U_sum, U_mean and the V_pi.  Returns |Aut(r)|."""
        p, names, aut = self.plan(k, edges)
        facs = [(us.MATRIX, 1.0, self.A.data_ptr()) if s == "A" else
                ((us.MATRIX, 1.0, self.B.data_ptr()) if self.B is not None else (us.COMPLEMENT, 1.0, self.A.data_ptr()))
                for s in names]
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        us.ustat_eval(p, self.X.data_ptr(), 0, self.n, 1, facs, self.ws.data_ptr(), self.ws.numel(), st,
                      out.data_ptr(), out.data_ptr() + 16)
        return aut

    def count(self, k, edges):
        """C(r, G) as a float (an exact integer for 0 / 1 input)."""
        p, _, _ = self.plan(k, edges)
        out = torch.empty(2 + p.info["n_parts"], dtype=torch.float64, device=self.device)
        aut = self.launch(k, edges, out)
        return float(out[0].item()) / aut
