"""Thin ctypes binding of the C ABI in include/ustat.h (argument marshalling only).

Every computation runs inside libustat.so; this module only converts Python
objects to the C structs and pointers, and torch tensors to device addresses.
Importing it loads the library; if the library is missing it raises, it never
falls back to another implementation.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libustat.so")

# status codes / kinds / modes (mirrors include/ustat.h)
USTAT_OK = 0
USTAT_ERR_INVALID_ARG = -1
USTAT_ERR_N_LT_M = -2
USTAT_ERR_TW_TOO_LARGE = -3
USTAT_ERR_WORKSPACE = -4
USTAT_ERR_NONFINITE = -5
USTAT_ERR_CUDA = -6
USTAT_ERR_DEVICE_TIMEOUT = -7
USTAT_ERR_UNSUPPORTED = -8

RBF, LINEAR, TANH_DOT, MATRIX, VECTOR, DIST, LOWRANK, COMPLEMENT, GRAM = 0, 1, 2, 3, 4, 5, 6, 7, 8
FP64, FP32, TF32, BF16X3, BF16X4, BF16X5 = 0, 1, 2, 3, 4, 5
PLAN_EXHAUSTIVE, PLAN_MINFILL = 0, 1
MAX_PARTS = 877   # Bell(7): partitions of the largest supported order m = 7
PRECISION = {"fp64": FP64, "fp32": FP32, "tf32": TF32, "bf16x3": BF16X3, "bf16x4": BF16X4, "bf16x5": BF16X5}

_P = ctypes.POINTER
_i = ctypes.c_int
_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_d = ctypes.c_double
_f = ctypes.c_float


class ustat_graph(ctypes.Structure):
    _fields_ = [("m", _i), ("n_edges", _i), ("edge_src", _P(_i)), ("edge_dst", _P(_i)),
                ("edge_factor", _P(_i)), ("n_unary", _i), ("unary_vertex", _P(_i)),
                ("unary_factor", _P(_i)), ("n_factors", _i), ("factor_kind", _P(_i))]


class ustat_options(ctypes.Structure):
    _fields_ = [("precision", _i), ("sparsify", _i), ("planner", _i), ("cse", _i)]


class ustat_factor(ctypes.Structure):
    _fields_ = [("kind", _i), ("param", _d), ("data", _vp)]


EXPORTS = {
    "ustat_plan": (_i, [_P(ustat_graph), _P(ustat_options), _P(_vp)]),
    "ustat_plan_destroy": (None, [_vp]),
    "ustat_plan_shard": (_i, [_P(ustat_graph), _P(ustat_options), _i, _i, _i64, _P(_i), _P(_vp)]),
    "ustat_plan_serialize": (_i, [_vp, _vp, _sz, _P(_sz)]),
    "ustat_plan_deserialize": (_i, [_vp, _sz, _P(_vp)]),
    "ustat_plan_info": (_i, [_vp, _P(_i), _P(_i), _P(_i), _P(_i), _P(_i), _P(_i), _P(_i), _P(_i)]),
    "ustat_plan_flops": (_i, [_vp, _i64, _P(_d), _P(_d)]),
    "ustat_plan_describe": (_i, [_vp, ctypes.c_char_p, _sz, _P(_sz)]),
    "ustat_workspace_bytes": (_i, [_vp, _i64, _i, _P(_sz)]),
    "ustat_status": (_i, [_vp, _vp, _P(_i)]),
    "ustat_factor_matrix": (_i, [_i, _d, _vp, _i64, _vp, _vp, _vp]),
    "ustat_lean_workspace_bytes": (_i, [_vp, _i64, _i, _i64, _P(_sz)]),
    "ustat_eval_lean": (_i, [_vp, _vp, _i, _i64, _i, _P(ustat_factor), _i, _i64, _vp, _sz, _vp, _vp, _vp]),
    "ustat_debug_set_wait": (_i, [ctypes.c_longlong, _i]),
    "ustat_scalar_count": (_i, [_vp, _P(_i)]),
    "ustat_eval_rows": (_i, [_vp, _i, _i, _vp, _i, _i64, _i, _P(ustat_factor), _i, _vp, _sz, _vp, _vp]),
    "ustat_combine": (_i, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "ustat_noalloc_status": (_i, [_vp, _P(_i)]),
    "ustat_eval": (_i, [_vp, _vp, _i, _i64, _i, _P(ustat_factor), _i, _vp, _sz, _vp, _vp, _vp]),
    "ustat_host_staging_bytes": (_i, [_vp, _i64, _i, _P(_sz)]),
    "ustat_eval_noalloc": (_i, [_vp, _vp, _i, _i64, _i, _P(ustat_factor), _i, _vp, _vp, _vp]),
    "ustat_eval_host": (_i, [_vp, _vp, _i, _i64, _i, _P(ustat_factor), _i, _vp, _sz, _vp, _P(_d), _P(_d)]),
    "ustat_eval_batch": (_i, [_vp, _P(_vp), _i, _P(_i64), _i, _i, _P(ustat_factor), _i, _vp, _sz, _vp,
                              _vp, _vp]),
    "ustat_batch_workspace_bytes": (_i, [_vp, _P(_i64), _i, _i, _P(_sz)]),
    "ustat_plan_set_variant": (_i, [_vp, _i, _i]),
    "ustat_batched_create": (_i, [_vp, _P(_i64), _i, _i, _i, _P(_vp)]),
    "ustat_batched_destroy": (None, [_vp]),
    "ustat_batched_workspace_bytes": (_i, [_vp, _P(_sz)]),
    "ustat_batched_info": (_i, [_vp, _P(_i), _P(_i)]),
    "ustat_batched_set_lanes": (_i, [_vp, _i]),
    "ustat_batched_set_grouped": (_i, [_vp, _i]),
    "ustat_batched_run": (_i, [_vp, _P(_vp), _i, _P(ustat_factor), _i, _vp, _sz, _vp, _vp, _vp]),
    "ustat_batched_capture": (_i, [_vp, _P(_vp), _i, _P(ustat_factor), _i, _vp, _sz, _vp, _vp, _vp]),
    "ustat_batched_replay": (_i, [_vp, _vp]),
    "ustat_batched_autotune": (_i, [_vp, _P(_vp), _i, _P(ustat_factor), _i, _vp, _sz, _vp, _vp, _vp, _P(_i),
                                    _P(_d)]),
    "ustat_order_candidates": (_i, [_P(ustat_graph), _P(ustat_options), _i64, _i, _i, _P(_i), _P(_i), _P(_f)]),
    "ustat_plan_contraction": (_i, [_P(ustat_graph), _P(ustat_options), _P(_i), _P(_vp)]),
    "ustat_order_features": (_i, [_P(ustat_graph), _P(ustat_options), _i64, _i, _P(_i), _P(_f)]),
    "ustat_plan_orders": (_i, [_vp, _P(_i)]),
    "ustat_mlp_param_count": (_i, [_i, _i]),
    "ustat_mlp_workspace_bytes": (_i, [_i, _i, _i, _P(_sz)]),
    "ustat_mlp_forward": (_i, [_vp, _i, _i, _vp, _i, _vp, _vp]),
    "ustat_mlp_loss_grad": (_i, [_vp, _i, _i, _vp, _vp, _i, _vp, _sz, _vp, _vp, _vp]),
    "ustat_mlp_adam": (_i, [_vp, _vp, _vp, _vp, _i, _f, _f, _f, _f, _i, _vp]),
    "ustat_rank_workspace_bytes": (_i, [_P(ustat_graph), _P(ustat_options), _P(_sz)]),
    "ustat_plan_learned": (_i, [_P(ustat_graph), _P(ustat_options), _i64, _vp, _i, _vp, _sz, _vp, _P(_vp)]),
    "ustat_profile_enable": (_i, [_i]),
    "ustat_profile_kinds": (_i, []),
    "ustat_profile_kind_name": (ctypes.c_char_p, [_i]),
    "ustat_profile_collect": (_i, [_P(_d), _P(_i)]),
    "ustat_last_cuda_error": (ctypes.c_char_p, []),
    "ustat_strerror": (ctypes.c_char_p, [_i]),
    "ustat_version": (ctypes.c_char_p, []),
}


def load(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError("libustat.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


class UstatError(RuntimeError):
    def __init__(self, code, where):
        msg = lib().ustat_strerror(code).decode()
        if code == USTAT_ERR_CUDA:
            msg += ": " + lib().ustat_last_cuda_error().decode()
        super().__init__("%s failed: %s (%d)" % (where, msg, code))
        self.code = code


def _check(rc, where):
    if rc != USTAT_OK:
        raise UstatError(rc, where)


def _iarr(vals):
    vals = list(vals)
    return (_i * max(1, len(vals)))(*vals)


class Plan:
    """Owns a ustat_plan_t.  ``graph`` has ``m``, ``edges`` [(a, b, f)], ``unary``
    [(v, f)]; ``factor_kinds`` lists the kind of every factor id.  With
    ``shard=(rank, n_shards, n)`` the plan is that rank's shard of the partition
    sum (ustat_plan_shard) and ``owner`` lists each partition's shard."""

    def __init__(self, graph, factor_kinds, precision="bf16x3", sparsify=False, planner=PLAN_EXHAUSTIVE,
                 cse=True, shard=None):
        self._keep = [
            _iarr(e[0] for e in graph.edges), _iarr(e[1] for e in graph.edges), _iarr(e[2] for e in graph.edges),
            _iarr(u[0] for u in graph.unary), _iarr(u[1] for u in graph.unary), _iarr(factor_kinds)]
        g = ustat_graph(graph.m, len(graph.edges), self._keep[0], self._keep[1], self._keep[2],
                        len(graph.unary), self._keep[3], self._keep[4], len(factor_kinds), self._keep[5])
        prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
        o = ustat_options(prec, int(bool(sparsify)), int(planner), int(bool(cse)))
        h = _vp()
        self.owner = None
        if shard is None:
            _check(lib().ustat_plan(ctypes.byref(g), ctypes.byref(o), ctypes.byref(h)), "ustat_plan")
        else:
            rank, n_shards, n = shard
            own = (_i * MAX_PARTS)()
            _check(lib().ustat_plan_shard(ctypes.byref(g), ctypes.byref(o), int(rank), int(n_shards), int(n), own,
                                          ctypes.byref(h)), "ustat_plan_shard")
        self.handle = h
        self.m = graph.m
        self.factor_kinds = list(factor_kinds)
        self.precision = prec
        self.info = self._info()
        if shard is not None:
            self.owner = list(own[:self.info["n_parts"]])

    @classmethod
    def from_handle(cls, handle, graph, factor_kinds, precision):
        """Wrap a ustat_plan_t made by another entry point (contraction or
        learned plans)."""
        self = cls.__new__(cls)
        self.handle = handle
        self.owner = None
        self.m = graph.m
        self.factor_kinds = list(factor_kinds)
        self.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        self.info = self._info()
        return self

    def _info(self):
        L = lib()
        nparts = _i()
        _check(L.ustat_plan_info(self.handle, ctypes.byref(nparts), None, None, None, None, None, None, None),
               "ustat_plan_info")
        k = nparts.value
        mu, tw, ev = (_i * k)(), (_i * k)(), (_i * k)()
        rgs = (_i * (k * self.m))()
        nops, ng, ng3 = _i(), _i(), _i()
        _check(L.ustat_plan_info(self.handle, ctypes.byref(nparts), mu, tw, rgs, ev, ctypes.byref(nops),
                                 ctypes.byref(ng), ctypes.byref(ng3)), "ustat_plan_info")
        return {"n_parts": k, "mu": list(mu), "tw": list(tw), "evaluated": list(ev),
                "rgs": [tuple(rgs[i * self.m:(i + 1) * self.m]) for i in range(k)],
                "n_ops": nops.value, "n_gemm": ng.value, "n_gemm3": ng3.value}

    def to_bytes(self):
        """The plan serialised (ustat_plan_serialize), for a cache."""
        need = _sz()
        _check(lib().ustat_plan_serialize(self.handle, None, 0, ctypes.byref(need)), "ustat_plan_serialize")
        buf = ctypes.create_string_buffer(need.value)
        _check(lib().ustat_plan_serialize(self.handle, buf, need.value, None), "ustat_plan_serialize")
        return buf.raw

    @classmethod
    def from_bytes(cls, data, graph, factor_kinds, precision):
        """A plan read back from to_bytes() (ustat_plan_deserialize)."""
        h = _vp()
        _check(lib().ustat_plan_deserialize(data, len(data), ctypes.byref(h)), "ustat_plan_deserialize")
        return cls.from_handle(h, graph, factor_kinds, precision)

    def flops(self, n):
        a, b = _d(), _d()
        _check(lib().ustat_plan_flops(self.handle, int(n), ctypes.byref(a), ctypes.byref(b)), "ustat_plan_flops")
        return a.value, b.value

    def describe(self):
        need = _sz()
        _check(lib().ustat_plan_describe(self.handle, None, 0, ctypes.byref(need)), "ustat_plan_describe")
        buf = ctypes.create_string_buffer(need.value)
        _check(lib().ustat_plan_describe(self.handle, buf, need.value, None), "ustat_plan_describe")
        return buf.value.decode()

    def set_variant(self, variant, size_class=-1):
        _check(lib().ustat_plan_set_variant(self.handle, int(size_class), int(variant)), "ustat_plan_set_variant")

    def workspace_bytes(self, n, d):
        s = _sz()
        _check(lib().ustat_workspace_bytes(self.handle, int(n), int(d), ctypes.byref(s)), "ustat_workspace_bytes")
        return s.value

    def host_staging_bytes(self, n, d):
        s = _sz()
        _check(lib().ustat_host_staging_bytes(self.handle, int(n), int(d), ctypes.byref(s)),
               "ustat_host_staging_bytes")
        return s.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.ustat_plan_destroy(h)
            self.handle = None


def graph_struct(graph, factor_kinds):
    """(ustat_graph, keep-alive arrays) for a synth.Graph-like object."""
    keep = [_iarr(e[0] for e in graph.edges), _iarr(e[1] for e in graph.edges), _iarr(e[2] for e in graph.edges),
            _iarr(u[0] for u in graph.unary), _iarr(u[1] for u in graph.unary), _iarr(factor_kinds)]
    g = ustat_graph(graph.m, len(graph.edges), keep[0], keep[1], keep[2], len(graph.unary), keep[3], keep[4],
                    len(factor_kinds), keep[5])
    return g, keep


def options_struct(precision="bf16x3", sparsify=False, planner=PLAN_EXHAUSTIVE, cse=True):
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    return ustat_options(prec, int(bool(sparsify)), int(planner), int(bool(cse)))


RANK_FEATURES = 20


def order_candidates(graph, factor_kinds, n, part=-1, precision="bf16x3", max_cand=100000):
    """Distinct elimination sequences of one partition (-1: the finest) with their
    features: (orders [count x m], features [count x RANK_FEATURES])."""
    g, keep = graph_struct(graph, factor_kinds)
    o = options_struct(precision)
    cnt = _i()
    cap = min(max_cand, 5040)   # at most m! <= 7! sequences
    orders = (_i * max(1, cap * graph.m))()
    feats = (_f * max(1, cap * RANK_FEATURES))()
    _check(lib().ustat_order_candidates(ctypes.byref(g), ctypes.byref(o), int(n), int(part), cap, ctypes.byref(cnt),
                                        orders, feats), "ustat_order_candidates")
    k = min(cnt.value, cap)
    return ([list(orders[i * graph.m:(i + 1) * graph.m]) for i in range(k)],
            [list(feats[i * RANK_FEATURES:(i + 1) * RANK_FEATURES]) for i in range(k)])


def order_features(graph, factor_kinds, n, order, part=-1, precision="bf16x3"):
    g, keep = graph_struct(graph, factor_kinds)
    o = options_struct(precision)
    oa = _iarr(list(order) + [-1] * (graph.m - len(order)))
    feats = (_f * RANK_FEATURES)()
    _check(lib().ustat_order_features(ctypes.byref(g), ctypes.byref(o), int(n), int(part), oa, feats),
           "ustat_order_features")
    return list(feats)


def plan_orders(plan):
    """The elimination order (block ids, -1 padded) the plan chose per partition."""
    k = plan.info["n_parts"]
    arr = (_i * (k * plan.m))()
    _check(lib().ustat_plan_orders(plan.handle, arr), "ustat_plan_orders")
    return [[v for v in arr[i * plan.m:(i + 1) * plan.m]] for i in range(k)]


def plan_contraction(graph, factor_kinds, order=None, precision="bf16x3", planner=PLAN_EXHAUSTIVE):
    g, keep = graph_struct(graph, factor_kinds)
    o = options_struct(precision, planner=planner)
    h = _vp()
    oa = _iarr(order) if order is not None else None
    _check(lib().ustat_plan_contraction(ctypes.byref(g), ctypes.byref(o), oa, ctypes.byref(h)),
           "ustat_plan_contraction")
    return Plan.from_handle(h, graph, factor_kinds, precision)


def rank_workspace_bytes(graph, factor_kinds, precision="bf16x3"):
    g, keep = graph_struct(graph, factor_kinds)
    o = options_struct(precision)
    s = _sz()
    _check(lib().ustat_rank_workspace_bytes(ctypes.byref(g), ctypes.byref(o), ctypes.byref(s)),
           "ustat_rank_workspace_bytes")
    return s.value


def plan_learned(graph, factor_kinds, n, params_ptr, hidden, ws_ptr, ws_bytes, stream, precision="bf16x3",
                 cse=True):
    g, keep = graph_struct(graph, factor_kinds)
    o = options_struct(precision, cse=cse)
    h = _vp()
    _check(lib().ustat_plan_learned(ctypes.byref(g), ctypes.byref(o), int(n), params_ptr, int(hidden), ws_ptr,
                                    ws_bytes, stream, ctypes.byref(h)), "ustat_plan_learned")
    return Plan.from_handle(h, graph, factor_kinds, precision)


def mlp_param_count(features, hidden):
    c = lib().ustat_mlp_param_count(int(features), int(hidden))
    if c < 0:
        raise UstatError(c, "ustat_mlp_param_count")
    return c


def mlp_workspace_bytes(features, hidden, rows):
    s = _sz()
    _check(lib().ustat_mlp_workspace_bytes(int(features), int(hidden), int(rows), ctypes.byref(s)),
           "ustat_mlp_workspace_bytes")
    return s.value


def mlp_forward(params_ptr, features, hidden, X_ptr, rows, y_ptr, stream):
    _check(lib().ustat_mlp_forward(params_ptr, features, hidden, X_ptr, rows, y_ptr, stream), "ustat_mlp_forward")


def mlp_loss_grad(params_ptr, features, hidden, X_ptr, t_ptr, rows, ws_ptr, ws_bytes, grad_ptr, loss_ptr, stream):
    _check(lib().ustat_mlp_loss_grad(params_ptr, features, hidden, X_ptr, t_ptr, rows, ws_ptr, ws_bytes, grad_ptr,
                                     loss_ptr, stream), "ustat_mlp_loss_grad")


def mlp_adam(params_ptr, grad_ptr, m_ptr, v_ptr, count, lr, beta1, beta2, eps, step, stream):
    _check(lib().ustat_mlp_adam(params_ptr, grad_ptr, m_ptr, v_ptr, count, lr, beta1, beta2, eps, step, stream),
           "ustat_mlp_adam")


def factor_array(factors):
    """factors: list of (kind, param, device_pointer_or_0)."""
    arr = (ustat_factor * len(factors))()
    for i, (k, p, ptr) in enumerate(factors):
        arr[i].kind = int(k)
        arr[i].param = float(p)
        arr[i].data = int(ptr) if ptr else None
    return arr


def ustat_eval(plan, X_ptr, x_dtype, n, d, factors, ws_ptr, ws_bytes, stream, U_ptr, V_ptr):
    fa = factor_array(factors)
    rc = lib().ustat_eval(plan.handle, X_ptr, x_dtype, n, d, fa, len(factors), ws_ptr, ws_bytes, stream,
                          U_ptr, V_ptr)
    _check(rc, "ustat_eval")


def version():
    """The library's version string (ustat_version)."""
    return lib().ustat_version().decode()


def status(ws_ptr, stream):
    """ustat_status: USTAT_OK, USTAT_ERR_DEVICE_TIMEOUT if a bounded device wait of
    the last evaluation in this workspace gave up, or USTAT_ERR_NONFINITE if it read
    a NaN or infinite input (waits for the stream)."""
    st = _i()
    _check(lib().ustat_status(ws_ptr, stream, ctypes.byref(st)), "ustat_status")
    return st.value


def lean_workspace_bytes(plan, n, d, panel_rows):
    """ustat_lean_workspace_bytes: the workspace of a memory-lean evaluation."""
    s = _sz()
    _check(lib().ustat_lean_workspace_bytes(plan.handle, int(n), int(d), int(panel_rows), ctypes.byref(s)),
           "ustat_lean_workspace_bytes")
    return s.value


def ustat_eval_lean(plan, X_ptr, x_dtype, n, d, factors, panel_rows, ws_ptr, ws_bytes, stream, U_ptr, V_ptr):
    """ustat_eval_lean: the evaluation with no n x n object stored (factor rows
    rebuilt in panels of panel_rows rows); device pointers as ustat_eval."""
    arr = factor_array(factors)
    _check(lib().ustat_eval_lean(plan.handle, X_ptr, int(x_dtype), int(n), int(d), arr, len(factors),
                                 int(panel_rows), ws_ptr, ws_bytes, stream, U_ptr, V_ptr), "ustat_eval_lean")


def factor_matrix(kind, param, data_ptr, n, F_ptr, ws_ptr, stream):
    """ustat_factor_matrix: the n x n float64 matrix of a DIST, LOWRANK, GRAM or
    COMPLEMENT factor (device pointers), built on the stream into F_ptr; the
    status word in ws_ptr (>= 256 bytes) is read by status()."""
    _check(lib().ustat_factor_matrix(int(kind), float(param), data_ptr, int(n), F_ptr, ws_ptr, stream),
           "ustat_factor_matrix")


def noalloc_status(stream):
    """ustat_noalloc_status: the status of the last ustat_eval_noalloc on the current
    device (waits for the stream)."""
    st = _i()
    _check(lib().ustat_noalloc_status(stream, ctypes.byref(st)), "ustat_noalloc_status")
    return st.value


def debug_set_wait(limit_cycles=0, stall_producer=False):
    """ustat_debug_set_wait: test hook of the bounded device waits (0, False = off)."""
    _check(lib().ustat_debug_set_wait(int(limit_cycles), 1 if stall_producer else 0), "ustat_debug_set_wait")


NOALLOC_MAX_BYTES = 64 * 1024 * 1024


def scalar_count(plan):
    """ustat_scalar_count: the length of a row shard's scalar array."""
    c = _i()
    _check(lib().ustat_scalar_count(plan.handle, ctypes.byref(c)), "ustat_scalar_count")
    return c.value


def ustat_eval_rows(plan, rank, n_ranks, X_ptr, x_dtype, n, d, factors, ws_ptr, ws_bytes, stream, scal_ptr):
    fa = factor_array(factors)
    rc = lib().ustat_eval_rows(plan.handle, rank, n_ranks, X_ptr, x_dtype, n, d, fa, len(factors), ws_ptr, ws_bytes,
                               stream, scal_ptr)
    _check(rc, "ustat_eval_rows")


def ustat_combine(plan, scal_ptr, n, stream, U_ptr, V_ptr):
    _check(lib().ustat_combine(plan.handle, scal_ptr, n, stream, U_ptr, V_ptr), "ustat_combine")


def ustat_eval_noalloc(plan, X_ptr, x_dtype, n, d, factors, stream, U_ptr, V_ptr):
    fa = factor_array(factors)
    rc = lib().ustat_eval_noalloc(plan.handle, X_ptr, x_dtype, n, d, fa, len(factors), stream, U_ptr, V_ptr)
    _check(rc, "ustat_eval_noalloc")


def ustat_eval_host(plan, X_host_ptr, x_dtype, n, d, factors, ws_ptr, ws_bytes, stream, U_host, V_host):
    fa = factor_array(factors)
    rc = lib().ustat_eval_host(plan.handle, X_host_ptr, x_dtype, n, d, fa, len(factors), ws_ptr, ws_bytes,
                               stream, U_host, V_host)
    _check(rc, "ustat_eval_host")


def ustat_eval_batch(plan, X_ptrs, x_dtype, ns, d, factors, ws_ptr, ws_bytes, stream, U_ptr, V_ptr):
    fa = factor_array(factors)
    xp = (_vp * len(X_ptrs))(*X_ptrs)
    na = (_i64 * len(ns))(*ns)
    rc = lib().ustat_eval_batch(plan.handle, xp, x_dtype, na, len(ns), d, fa, len(factors), ws_ptr, ws_bytes,
                                stream, U_ptr, V_ptr)
    _check(rc, "ustat_eval_batch")


def batch_workspace_bytes(plan, ns, d):
    s = _sz()
    na = (_i64 * len(ns))(*ns)
    _check(lib().ustat_batch_workspace_bytes(plan.handle, na, len(ns), d, ctypes.byref(s)),
           "ustat_batch_workspace_bytes")
    return s.value


class Batched:
    """Owns a ustat_batched_t: one plan over many samples of uneven size, run on
    several streams, optionally captured into one CUDA graph.  Pointers are plain
    integers (device addresses)."""

    def __init__(self, plan, ns, d, max_lanes=0):
        self.plan = plan   # keeps the plan alive
        self.count = len(ns)
        self.ns = [int(v) for v in ns]
        na = (_i64 * self.count)(*self.ns)
        h = _vp()
        _check(lib().ustat_batched_create(plan.handle, na, self.count, int(d), int(max_lanes), ctypes.byref(h)),
               "ustat_batched_create")
        self.handle = h

    def workspace_bytes(self):
        s = _sz()
        _check(lib().ustat_batched_workspace_bytes(self.handle, ctypes.byref(s)), "ustat_batched_workspace_bytes")
        return s.value

    def info(self):
        lanes = _i()
        lane_of = (_i * self.count)()
        _check(lib().ustat_batched_info(self.handle, ctypes.byref(lanes), lane_of), "ustat_batched_info")
        return lanes.value, list(lane_of)

    def set_lanes(self, lanes):
        _check(lib().ustat_batched_set_lanes(self.handle, int(lanes)), "ustat_batched_set_lanes")

    def set_grouped(self, grouped=True):
        """ustat_batched_set_grouped: one persistent launch per product step over
        all samples' tiles (bf16x3); the workspace grows to one region per sample."""
        _check(lib().ustat_batched_set_grouped(self.handle, 1 if grouped else 0), "ustat_batched_set_grouped")

    def _args(self, X_ptrs, factors):
        if len(X_ptrs) != self.count:
            raise ValueError("one X pointer per sample")
        return (_vp * self.count)(*X_ptrs), factor_array(factors)

    def run(self, X_ptrs, x_dtype, factors, ws_ptr, ws_bytes, stream, U_ptr, V_ptr):
        xp, fa = self._args(X_ptrs, factors)
        _check(lib().ustat_batched_run(self.handle, xp, x_dtype, fa, len(factors), ws_ptr, ws_bytes, stream, U_ptr,
                                       V_ptr), "ustat_batched_run")

    def capture(self, X_ptrs, x_dtype, factors, ws_ptr, ws_bytes, stream, U_ptr, V_ptr):
        xp, fa = self._args(X_ptrs, factors)
        _check(lib().ustat_batched_capture(self.handle, xp, x_dtype, fa, len(factors), ws_ptr, ws_bytes, stream,
                                           U_ptr, V_ptr), "ustat_batched_capture")

    def replay(self, stream):
        _check(lib().ustat_batched_replay(self.handle, stream), "ustat_batched_replay")

    def autotune(self, X_ptrs, x_dtype, factors, ws_ptr, ws_bytes, stream, U_ptr, V_ptr):
        xp, fa = self._args(X_ptrs, factors)
        lanes, ms = _i(), _d()
        _check(lib().ustat_batched_autotune(self.handle, xp, x_dtype, fa, len(factors), ws_ptr, ws_bytes, stream,
                                            U_ptr, V_ptr, ctypes.byref(lanes), ctypes.byref(ms)),
               "ustat_batched_autotune")
        return lanes.value, ms.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.ustat_batched_destroy(h)
            self.handle = None


def profile_enable(on: bool):
    _check(lib().ustat_profile_enable(int(bool(on))), "ustat_profile_enable")


def profile_collect():
    """Returns {kind_name: (total_ms, launches)} for the operations recorded since
    the last call (only kinds that ran)."""
    L = lib()
    k = L.ustat_profile_kinds()
    ms = (_d * k)()
    cnt = (_i * k)()
    _check(L.ustat_profile_collect(ms, cnt), "ustat_profile_collect")
    return {L.ustat_profile_kind_name(i).decode(): (ms[i], cnt[i]) for i in range(k) if cnt[i]}
