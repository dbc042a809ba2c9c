"""Higher-order influence function (HOIF) chain U-statistics (the example of
Section 4.1).  For an unconfounded sample X_i = (Z_i, A_i, Y_i) with a
dictionary phi, the estimator's terms are U-statistics of the chain kernels

    h_2(X_1, X_2)     = f(X_1, X_2)
    h_j(X_1 .. X_j)   = g(X_1, X_2) g(X_2, X_3) ... g(X_{j-2}, X_{j-1}) f(X_{j-1}, X_j),

    g(X_a, X_b) = A_a phi(Z_a)' A_b phi(Z_b),   f(X_a, X_b) = A_a phi(Z_a)' phi(Z_b) Y_b,

a chain of j - 1 pairwise factors (signature ((1, 2), ..., (j - 1, j))).  The
factors G = Psi Psi' and F = Psi Theta', with Psi_i = A_i phi(Z_i) and
Theta_i = phi(Z_i) Y_i, enter the engine as a GRAM factor (symmetric: the
planner reads it untransposed and computes only the upper tiles of symmetric
products) and a LOWRANK factor: only the n x k terms Psi and Theta are
uploaded, and the library builds the n x n matrices on the device (the
tensorization step); every U_sum is then one exact evaluation (all Bell(j)
restricted V-statistics and the Moebius combination) on the device.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ustat as us


class _Graph:
    def __init__(self, m, edges):
        self.m = m
        self.edges = edges
        self.unary = []


def chain_graph(j):
    """The chain 0 - ... - (j-1): factor 0 = g on the first j - 2 edges, the
    last factor id = f on the last edge (for j = 2: f alone, id 0)."""
    if j < 2:
        raise ValueError("chains have j >= 2")
    if j == 2:
        return _Graph(2, [(0, 1, 0)]), ["f"]
    return _Graph(j, [(v, v + 1, 0) for v in range(j - 2)] + [(j - 2, j - 1, 1)]), ["g", "f"]


def factor_terms(phi, A, Y):
    """The data of the two factors (float64): Psi (n x k) for the GRAM factor
    g = Psi Psi', and [Psi | Theta] (n x 2k) for the LOWRANK factor f = Psi Theta'."""
    phi = np.asarray(phi, dtype=np.float64)
    Psi = np.asarray(A, dtype=np.float64)[:, None] * phi
    Theta = phi * np.asarray(Y, dtype=np.float64)[:, None]
    return np.ascontiguousarray(Psi), np.ascontiguousarray(np.hstack([Psi, Theta]))


def factor_matrices(phi, A, Y):
    """G = Psi Psi' and F = Psi Theta' (float64, n x n), formed on the host: for
    callers that hold the matrices themselves (the engine builds them from
    factor_terms)."""
    TG, TF = factor_terms(phi, A, Y)
    k = TG.shape[1]
    return TG @ TG.T, TF[:, :k] @ TF[:, k:].T


class HoifChains:
    """Device copies of the factor terms (n x k and n x 2k), one plan per chain
    length, one workspace; the library builds G and F on the device in every
    evaluation."""

    def __init__(self, n, k=16, orders=(2, 3, 4, 5, 6, 7), precision="bf16x4", device="cuda:0"):
        self.n = n
        self.k = k
        self.device = torch.device(device)
        self.orders = list(orders)
        self.plans = {}
        for j in self.orders:
            g, names = chain_graph(j)
            kinds = [us.GRAM if s == "g" else us.LOWRANK for s in names]
            self.plans[j] = (us.Plan(g, kinds, precision=precision), names)
        need = max(256, max(p.workspace_bytes(n, 1) for p, _ in self.plans.values()))
        self.ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        self.TG = torch.empty((n, k), dtype=torch.float64, device=self.device)
        self.TF = torch.empty((n, 2 * k), dtype=torch.float64, device=self.device)
        self.X = torch.zeros((n, 1), dtype=torch.float64, device=self.device)
        self.out = {j: torch.empty(2 + p.info["n_parts"], dtype=torch.float64, device=self.device)
                    for j, (p, _) in self.plans.items()}

    def set(self, TG, TF, non_blocking=False):
        """The factor terms Psi (n x k) and [Psi | Theta] (n x 2k) (numpy or host /
        device tensors, float64)."""
        for dst, src in ((self.TG, TG), (self.TF, TF)):
            if not isinstance(src, torch.Tensor):
                src = torch.from_numpy(np.ascontiguousarray(src, dtype=np.float64))
            dst.copy_(src, non_blocking=non_blocking)

    def launch(self, j, stream=None):
        """Enqueue U(h_j): out[j] = U_sum, U_mean, V_pi."""
        p, names = self.plans[j]
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        facs = [(us.GRAM, float(self.k), self.TG.data_ptr()) if s == "g" else
                (us.LOWRANK, float(self.k), self.TF.data_ptr()) for s in names]
        o = self.out[j]
        us.ustat_eval(p, self.X.data_ptr(), 0, self.n, 1, facs, self.ws.data_ptr(), self.ws.numel(), st,
                      o.data_ptr(), o.data_ptr() + 16)

    def evaluate(self, phi, A, Y):
        """U_sum of every chain order: {j: U_sum}."""
        self.set(*factor_terms(phi, A, Y))
        for j in self.orders:
            self.launch(j)
        return {j: float(self.out[j][0].item()) for j in self.orders}
