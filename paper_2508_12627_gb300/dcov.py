"""Squared distance covariance as a combination of exact U-statistics (the
distance-covariance example of Section 4.3).  With a_ij = ||x_i - x_j|| and
b_ij = ||y_i - y_j||, the paper writes dCov^2 as the order-4 U-statistic

    dCov^2 = 1/(n)_4 * sum over ordered distinct (i, j, k, l) of
             a_ij b_kl + a_ij b_ij - a_ij b_ik - a_ij b_jl .

A product that does not touch every one of the four indices sums the untouched
ones out over the values distinct from the others: a_ij b_ij leaves two
(a factor (n - 2)(n - 3)), a_ij b_ik and a_ij b_jl leave one (a factor n - 3).
So dCov^2 is a combination of four kernel graphs, each evaluated exactly by the
engine from the two distance matrices (MATRIX factors):

    (n)_4 dCov^2 = U_4[a_01 b_23] + (n-2)(n-3) U_2[a_01 b_01]
                   - (n-3) U_3[a_01 b_02] - (n-3) U_3[a_01 b_12]

where U_k[.] is the sum over ordered distinct k-tuples.  The distance matrices
are built on the device from the caller's samples X (n x p) and Y (n x q) by
ustat_factor_matrix (the DIST factor: float64 coordinate differences), once per
sample, and enter the four evaluations as MATRIX factors; the four U_sums come
back to the host, which forms the combination (four scalars) with a compensated
sum.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import ustat as us

# (coefficient in n, order k, edges (a, b, factor): factor 0 = a, 1 = b)
TERMS = [
    (lambda n: 1.0, 4, [(0, 1, 0), (2, 3, 1)]),
    (lambda n: float((n - 2) * (n - 3)), 2, [(0, 1, 0), (0, 1, 1)]),
    (lambda n: -float(n - 3), 3, [(0, 1, 0), (0, 2, 1)]),
    (lambda n: -float(n - 3), 3, [(0, 1, 0), (1, 2, 1)]),
]


class _Graph:
    def __init__(self, m, edges):
        self.m = m
        self.edges = edges
        self.unary = []


def distances(Z):
    """n x n Euclidean distances between the rows of Z (float64), from the
    coordinate differences (no cancellation), a block of rows at a time: the
    matrix the DIST factor builds on the device, for callers that want it."""
    Z = np.asarray(Z, dtype=np.float64)
    if Z.ndim == 1:
        Z = Z[:, None]
    n, p = Z.shape
    out = np.empty((n, n))
    rows = max(1, (1 << 24) // max(1, n * p))
    for r0 in range(0, n, rows):
        D = Z[r0:r0 + rows, None, :] - Z[None, :, :]
        out[r0:r0 + rows] = np.sqrt(np.einsum("ijk,ijk->ij", D, D))
    return out


class DCov2:
    """The four plans for sample size n (MATRIX factors), distance-matrix buffers,
    one workspace."""

    def __init__(self, n, precision="fp64", device="cuda:0"):
        if n < 4:
            raise ValueError("dCov^2 needs n >= 4")
        self.n = n
        self.device = torch.device(device)
        self.plans = [us.Plan(_Graph(k, e), [us.MATRIX, us.MATRIX], precision=precision) for _, k, e in TERMS]
        self.coef = [c(n) for c, _, _ in TERMS]
        need = max(256, max(p.workspace_bytes(n, 1) for p in self.plans))
        self.ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        self.fws = torch.empty(256, dtype=torch.uint8, device=self.device)   # status word of the builds
        self.a = self.b = None
        self.Da = torch.empty((n, n), dtype=torch.float64, device=self.device)
        self.Db = torch.empty_like(self.Da)
        self.X = torch.zeros((n, 1), dtype=torch.float64, device=self.device)
        self.out = [torch.empty(2 + p.info["n_parts"], dtype=torch.float64, device=self.device) for p in self.plans]

    def _dev(self, Z):
        if not isinstance(Z, torch.Tensor):
            Z = torch.from_numpy(np.ascontiguousarray(Z, dtype=np.float64))
        if Z.dim() == 1:
            Z = Z[:, None]
        return Z.to(device=self.device, dtype=torch.float64).contiguous()

    def set(self, X, Y):
        """The paired samples (n x p and n x q; numpy or tensors) on the device."""
        self.a, self.b = self._dev(X), self._dev(Y)

    def distance(self, Z, D=None, stream=None):
        """Enqueue D = the n x n distances between the rows of the device sample Z
        (n x p float64, contiguous) into D (default: a new device tensor); returns D."""
        if Z.dim() != 2 or Z.shape[0] != self.n or Z.dtype != torch.float64 or not Z.is_contiguous():
            raise ValueError("Z must be a contiguous n x p float64 device tensor")
        D = torch.empty((self.n, self.n), dtype=torch.float64, device=self.device) if D is None else D
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        us.factor_matrix(us.DIST, float(Z.shape[1]), Z.data_ptr(), self.n, D.data_ptr(), self.fws.data_ptr(), st)
        return D

    def launch_matrices(self, Da, Db, out=None, stream=None):
        """Enqueue the four U-statistics of the distance matrices Da and Db (device
        n x n float64) into out (four float64 device tensors of 2 + Bell(k);
        default: this object's)."""
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        facs = [(us.MATRIX, 1.0, Da.data_ptr()), (us.MATRIX, 1.0, Db.data_ptr())]
        for p, o in zip(self.plans, self.out if out is None else out):
            us.ustat_eval(p, self.X.data_ptr(), 0, self.n, 1, facs, self.ws.data_ptr(), self.ws.numel(), st,
                          o.data_ptr(), o.data_ptr() + 16)

    def launch(self, a=None, b=None, out=None, stream=None):
        """Enqueue dCov^2 of the device samples a (n x p) and b (n x q), float64
        (default: the copies made by set()): their distance matrices into this
        object's buffers, then the four U-statistics into out."""
        a = self.a if a is None else a
        b = self.b if b is None else b
        self.distance(a, self.Da, stream)
        self.distance(b, self.Db, stream)
        self.launch_matrices(self.Da, self.Db, out, stream)

    def capture(self, enqueue):
        """One CUDA graph of the launches that enqueue() makes on the current
        stream (for instance the distance matrices of several samples and the
        evaluations of many pairs).  At n in the hundreds every kernel takes a few
        microseconds and an eager sequence is bound by launch latency; the graph
        replays the same kernels, on the buffers' current contents, with one
        launch.  enqueue() runs once eagerly first, outside the capture, so that
        every lazily prepared resource of the plans exists before capturing."""
        cur = torch.cuda.current_stream(self.device)
        side = torch.cuda.Stream(self.device)
        side.wait_stream(cur)
        with torch.cuda.stream(side):
            enqueue()
        cur.wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side, capture_error_mode="thread_local"):
            enqueue()
        return graph

    def combine(self, U_sums):
        """dCov^2 from the four U_sums, and the scale sum |coef U| / (n)_4 against
        which its rounding is judged."""
        ff = float(math.perm(self.n, 4))
        terms = [c * u for c, u in zip(self.coef, U_sums)]
        return math.fsum(terms) / ff, math.fsum(abs(t) for t in terms) / ff

    def evaluate(self, X, Y):
        """dCov^2(X, Y) for n paired samples (rows); returns (value, scale)."""
        self.set(X, Y)
        self.launch()
        return self.combine([float(o[0].item()) for o in self.out])
