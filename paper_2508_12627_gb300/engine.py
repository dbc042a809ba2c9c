"""Torch-facing convenience layer over the C ABI: device buffers come from torch,
the stream is torch's current stream, and every computation runs in libustat.so.

    eng = Engine(graph, factors, precision="bf16x3")
    out = eng.evaluate(X)          # X: torch tensor on the GPU or a numpy array
    out["U_sum"], out["U_mean"], out["V"]

``factors`` is a list of objects with ``kind``, ``param`` and ``data`` (the
TANH_DOT weight vector, the MATRIX / VECTOR values as arrays); their data is
copied to the device once per sample size.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ustat as us


class Engine:
    def __init__(self, graph, factors, precision="bf16x3", sparsify=False, planner=us.PLAN_EXHAUSTIVE, cse=True,
                 device="cuda:0", shard=None, plan_cache=None):
        """``shard=(rank, n_shards, n)``: evaluate only this rank's share of the
        partition sum (ustat_plan_shard); ``evaluate_shards`` then sums the
        ranks' results.  ``plan_cache``: a directory where plans are kept as
        serialised bytes, keyed by everything that determines them."""
        self.graph = graph
        self.factors = list(factors)
        self.device = torch.device(device)
        kinds = [f.kind for f in self.factors]
        self.plan = None
        self.plan_cached = False
        path = None
        if plan_cache is not None and shard is None:
            import hashlib
            import os
            key = repr((graph.m, sorted(tuple(e) for e in graph.edges), sorted(tuple(u) for u in graph.unary), kinds,
                        precision, bool(sparsify), int(planner), bool(cse), us.version()))
            os.makedirs(plan_cache, exist_ok=True)
            path = os.path.join(plan_cache, hashlib.sha256(key.encode()).hexdigest()[:32] + ".plan")
            if os.path.exists(path):
                with open(path, "rb") as f:
                    self.plan = us.Plan.from_bytes(f.read(), graph, kinds, precision)
                self.plan_cached = True
        if self.plan is None:
            self.plan = us.Plan(graph, kinds, precision=precision, sparsify=sparsify, planner=planner, cse=cse,
                                shard=shard)
            if path is not None:
                with open(path, "wb") as f:
                    f.write(self.plan.to_bytes())
        self.n_parts = self.plan.info["n_parts"]
        self._ws = None
        self._fdev = {}

    # device copies of factor data, keyed by n (MATRIX / VECTOR data depend on n)
    def factor_tuples(self, n):
        out = []
        keep = []
        for f in self.factors:
            ptr = 0
            if f.data is not None:
                key = (id(f), n)
                t = self._fdev.get(key)
                if t is None:
                    t = torch.as_tensor(np.ascontiguousarray(f.data, dtype=np.float64), device=self.device)
                    self._fdev[key] = t
                keep.append(t)
                ptr = t.data_ptr()
            out.append((f.kind, f.param, ptr))
        return out

    def workspace(self, nbytes):
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def to_device(self, X):
        if isinstance(X, torch.Tensor):
            X = X.to(self.device)
        else:
            X = torch.as_tensor(np.ascontiguousarray(X), device=self.device)
        if X.dtype not in (torch.float64, torch.float32):
            X = X.to(torch.float64)
        return X.contiguous()

    def launch(self, X, out, stream=None):
        """Enqueue one evaluation; ``out`` is a float64 device tensor of 2 + n_parts."""
        n, d = X.shape
        ws = self.workspace(self.plan.workspace_bytes(n, d))
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        us.ustat_eval(self.plan, X.data_ptr(), 0 if X.dtype == torch.float64 else 1, n, d, self.factor_tuples(n),
                      ws.data_ptr(), ws.numel(), st, out.data_ptr(), out.data_ptr() + 16)

    def evaluate(self, X):
        X = self.to_device(X)
        out = torch.empty(2 + self.n_parts, dtype=torch.float64, device=self.device)
        self.launch(X, out)
        o = out.cpu().numpy()
        return {"U_sum": float(o[0]), "U_mean": float(o[1]), "V": o[2:].copy()}

    def evaluate_lean(self, X, panel_rows=4096):
        """The memory-lean evaluation (ustat_eval_lean): no n x n factor or product is
        stored; the factor rows are rebuilt from X in panels of panel_rows rows."""
        X = self.to_device(X)
        n, d = X.shape
        ws = self.workspace(us.lean_workspace_bytes(self.plan, n, d, panel_rows))
        out = torch.empty(2 + self.n_parts, dtype=torch.float64, device=self.device)
        st = torch.cuda.current_stream(self.device).cuda_stream
        us.ustat_eval_lean(self.plan, X.data_ptr(), 0 if X.dtype == torch.float64 else 1, n, d,
                           self.factor_tuples(n), panel_rows, ws.data_ptr(), ws.numel(), st, out.data_ptr(),
                           out.data_ptr() + 16)
        o = out.cpu().numpy()
        return {"U_sum": float(o[0]), "U_mean": float(o[1]), "V": o[2:].copy()}

    @staticmethod
    def reduce_shards(out, group=None):
        """The exchange step of a sharded evaluation: ``out`` (2 + Bell(m)
        float64: U_sum, U_mean, V) holds this rank's partitions and zeros
        elsewhere; one all-reduce (sum) over the ranks of ``group`` gives every
        rank the full result, since U_sum, U_mean and each V_pi are linear in
        the per-partition terms (Lemma "Decomposition of U-Statistic into
        V-Statistics")."""
        import torch.distributed as dist
        dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
        o = out.cpu().numpy()
        return {"U_sum": float(o[0]), "U_mean": float(o[1]), "V": o[2:].copy()}

    def evaluate_shards(self, X, group=None):
        """This rank's shard on its GPU, then the all-reduce of the 2 + Bell(m)
        results (NCCL for device tensors)."""
        X = self.to_device(X)
        out = torch.empty(2 + self.n_parts, dtype=torch.float64, device=self.device)
        self.launch(X, out)
        return self.reduce_shards(out, group)

    def scalars_rows(self, X, rank, n_ranks):
        """This rank's row shard of one evaluation (ustat_eval_rows): a float64 device
        tensor of the plan's scalars, which sums over the ranks to the whole
        evaluation's scalars."""
        X = self.to_device(X)
        n, d = X.shape
        ws = self.workspace(self.plan.workspace_bytes(n, d))
        scal = torch.zeros(max(1, us.scalar_count(self.plan)), dtype=torch.float64, device=self.device)
        st = torch.cuda.current_stream(self.device).cuda_stream
        us.ustat_eval_rows(self.plan, rank, n_ranks, X.data_ptr(), 0 if X.dtype == torch.float64 else 1, n, d,
                           self.factor_tuples(n), ws.data_ptr(), ws.numel(), st, scal.data_ptr())
        return scal

    def combine(self, scal, n):
        """U and V from a plan's (summed) scalars (ustat_combine)."""
        out = torch.empty(2 + self.n_parts, dtype=torch.float64, device=self.device)
        st = torch.cuda.current_stream(self.device).cuda_stream
        us.ustat_combine(self.plan, scal.data_ptr(), n, st, out.data_ptr(), out.data_ptr() + 16)
        o = out.cpu().numpy()
        return {"U_sum": float(o[0]), "U_mean": float(o[1]), "V": o[2:].copy()}

    @staticmethod
    def reduce_row_scalars(scal, group=None):
        """The exchange step of a row-sharded evaluation: one all-reduce (sum) of the
        ranks' scalar arrays (NCCL for device tensors)."""
        import torch.distributed as dist
        dist.all_reduce(scal, op=dist.ReduceOp.SUM, group=group)
        return scal

    def evaluate_rows(self, X, group=None):
        """One evaluation row-sharded over the ranks of ``group`` (one GPU each):
        this rank's share, the all-reduce of the scalars, the combination."""
        import torch.distributed as dist
        scal = self.scalars_rows(X, dist.get_rank(group), dist.get_world_size(group))
        self.reduce_row_scalars(scal, group)
        return self.combine(scal, X.shape[0])

    def evaluate_host(self, X_host_pinned, U_host, V_host):
        """End-to-end call with host input and outputs (ustat_eval_host):
        X_host_pinned is a pinned torch CPU tensor, U_host / V_host ctypes arrays."""
        n, d = X_host_pinned.shape
        need = self.plan.workspace_bytes(n, d) + self.plan.host_staging_bytes(n, d)
        ws = self.workspace(need)
        st = torch.cuda.current_stream(self.device).cuda_stream
        us.ustat_eval_host(self.plan, X_host_pinned.data_ptr(), 0 if X_host_pinned.dtype == torch.float64 else 1,
                           n, d, self.factor_tuples(n), ws.data_ptr(), ws.numel(), st, U_host, V_host)
