"""ctypes front end of the brute-force C evaluator (oracle/brute.c).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  ``build()`` compiles the C
file with gcc into oracle/_build/; the CUDA library never loads it.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess

import numpy as np

from . import ustat_oracle as uo

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brute.c")
_OUT = os.path.join(_HERE, "_build", "liboracle_brute.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", _OUT, _SRC])
    return _OUT


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        _lib.oracle_brute_u_patterns.argtypes = [
            ctypes.c_int64, ctypes.c_int, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int),
            P(ctypes.c_int), P(P(ctypes.c_double)), P(ctypes.c_int), ctypes.c_int,
            P(ctypes.c_double)]
        _lib.oracle_brute_v.argtypes = [
            ctypes.c_int64, ctypes.c_int, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int),
            P(ctypes.c_int), P(P(ctypes.c_double)), P(ctypes.c_int), P(ctypes.c_double)]
    return _lib


def _marshal(sig, tensors):
    K = len(sig)
    arity = (ctypes.c_int * K)()
    i0 = (ctypes.c_int * K)()
    i1 = (ctypes.c_int * K)()
    keep = []
    ptrs = (ctypes.POINTER(ctypes.c_double) * K)()
    for k, (tup, T) in enumerate(zip([s[0] for s in sig], tensors)):
        a = np.ascontiguousarray(T, dtype=np.float64)
        keep.append(a)
        arity[k] = len(tup)
        i0[k] = tup[0]
        i1[k] = tup[1] if len(tup) == 2 else 0
        ptrs[k] = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return K, arity, i0, i1, ptrs, keep


def equality_patterns(m: int):
    """Every partition of [m], found as the equality pattern (first-occurrence
    labelling) of some tuple in [m]^m; sorted.  Independent of the oracle's own
    partition generator."""
    pats = set()
    for t in itertools.product(range(m), repeat=m):
        first = {}
        pats.add(tuple(first.setdefault(x, len(first)) for x in t))
    return sorted(pats)


def brute_all(graph, factors, X, sparse: bool = False):
    """Brute force over [n]^m.  Returns dict with
    ``U_pattern`` (restricted U-statistic per partition, in set_partitions order),
    ``U_sum`` (pattern of the finest partition), ``V`` (V_pi per partition straight
    from its V-set) and ``rgs``."""
    lib = _load()
    X = np.asarray(X)
    n = X.shape[0]
    m = graph.m
    sig = uo.signature(graph)
    T = uo.tensorize(graph, factors, X)
    if sparse:
        T = {f: uo.sparsify(a) for f, a in T.items()}
    tensors = [T[f] for _, f in sig]
    K, arity, i0, i1, ptrs, keep = _marshal(sig, tensors)
    parts = equality_patterns(m)
    code_to_idx = (ctypes.c_int * (m ** m))(*([-1] * (m ** m)))
    for p, rgs in enumerate(parts):
        code_to_idx[sum(b * m ** i for i, b in enumerate(rgs))] = p
    U = (ctypes.c_double * len(parts))()
    rc = lib.oracle_brute_u_patterns(n, m, K, arity, i0, i1, ptrs, code_to_idx, len(parts), U)
    assert rc == 0
    V = []
    for rgs in parts:
        v = ctypes.c_double()
        r = (ctypes.c_int * m)(*rgs)
        rc = lib.oracle_brute_v(n, m, K, arity, i0, i1, ptrs, r, ctypes.byref(v))
        assert rc == 0
        V.append(v.value)
    finest = tuple(range(m))
    return {"U_pattern": list(U), "U_sum": U[parts.index(finest)], "V": V, "rgs": parts}
