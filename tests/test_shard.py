"""Sharding one sample's partition sum over ranks (ustat_plan_shard): every
evaluated partition belongs to exactly one shard, all ranks compute the same
assignment, shared contractions are not repeated, and the ranks' results summed
(the one exchange step) give the full U and V.  Host-side checks run on CPU
(gloo ranks for the exchange); the GPU test runs every shard on one GPU."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from oracle import ustat_oracle as uo
from tests.conftest import ROOT

WORKLOADS = ["triangle_rbf", "c4_rbf", "path5_chord_linear_tanh", "k4_cycle_rbf"]
FULL_N = {"triangle_rbf": 200, "c4_rbf": 4096, "path5_chord_linear_tanh": 16384, "k4_cycle_rbf": 1024}


@pytest.fixture(scope="module")
def us():
    from paper_2508_12627_gb300 import build
    build.build()
    from paper_2508_12627_gb300 import ustat
    return ustat


def _shards(us, name, N, **kw):
    w = synth.workload(name, 8)
    kinds = [f.kind for f in w.factors]
    return w, [us.Plan(w.graph, kinds, shard=(r, N, FULL_N[name]), **kw) for r in range(N)]


@pytest.mark.parametrize("sparsify", [False, True])
@pytest.mark.parametrize("N", [1, 2, 3, 8])
@pytest.mark.parametrize("name", WORKLOADS)
def test_shards_cover_each_partition_once(us, name, N, sparsify):
    w, plans = _shards(us, name, N, sparsify=sparsify)
    full = us.Plan(w.graph, [f.kind for f in w.factors], sparsify=sparsify)
    owner = plans[0].owner
    assert all(p.owner == owner for p in plans)                  # one assignment on every rank
    ev_full = full.info["evaluated"]
    for i, o in enumerate(owner):
        assert (o >= 0) == bool(ev_full[i])                       # sparsified partitions belong to no shard
        assert o < N
        for r, p in enumerate(plans):
            assert p.info["evaluated"][i] == int(o == r)
    for p in plans:                                               # same partitions, mu and treewidths
        assert p.info["mu"] == full.info["mu"] and p.info["rgs"] == full.info["rgs"]
    # no n^4 step is repeated, and the few n^3 products and n^2 passes that two
    # shards both compute add at most 0.1 % to the full plan's flops
    n = FULL_N[name]
    tot = sum(p.flops(n)[0] for p in plans)
    assert tot <= full.flops(n)[0] * 1.001
    assert sum(p.info["n_gemm3"] for p in plans) == full.info["n_gemm3"]


def test_independent_contractions_are_balanced(us):
    # K4 + cycle: 18 distinct n^4 steps over 8 shards; path + chord: two
    # independent halves of equal cost
    _, plans = _shards(us, "k4_cycle_rbf", 8)
    f = [p.flops(1024)[0] for p in plans]
    assert max(f) <= 1.35 * sum(f) / 8
    _, plans = _shards(us, "path5_chord_linear_tanh", 2)
    f = [p.flops(16384)[0] for p in plans]
    assert max(f) <= 1.01 * sum(f) / 2


def test_shard_arguments_are_checked(us):
    g = synth.cycle4_graph()
    for bad in [(2, 2, 64), (-1, 2, 64), (0, 0, 64), (0, 2, 0)]:
        with pytest.raises(us.UstatError):
            us.Plan(g, [uo.RBF], shard=bad)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    from paper_2508_12627_gb300 import ustat as us
    from paper_2508_12627_gb300.engine import Engine
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.workload("k4_cycle_rbf", 9)
    plan = us.Plan(w.graph, [f.kind for f in w.factors], shard=(rank, world, 1024))
    # this rank's partial result, its partitions' V from the oracle (no GPU here)
    parts = uo.set_partitions(w.graph.m)
    mine = [p for p, o in zip(parts, plan.owner) if o == rank]
    part = uo.ustat(w.graph, w.factors, w.X, partitions=mine)
    V = np.zeros(len(parts))
    for rgs, v in zip(mine, part["V"]):
        V[parts.index(rgs)] = v
    out = torch.as_tensor(np.concatenate([[part["U_sum"], part["U_mean"]], V]))
    res = Engine.reduce_shards(out)
    dist.destroy_process_group()
    q.put((rank, len(mine), res["U_sum"], res["U_mean"], res["V"].tolist()))


def test_two_gloo_ranks_sum_their_shards():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert res[0][1] > 0 and res[1][1] > 0 and res[0][1] + res[1][1] == 203
    w = synth.workload("k4_cycle_rbf", 9)
    ref = uo.ustat(w.graph, w.factors, w.X)
    a = uo.ustat(w.graph, w.factors, w.X, absolute=True)
    uabs = float(np.abs(np.array(a["mu"], dtype=float)) @ np.array(a["V"]))
    for _, _, u_sum, u_mean, V in res:
        assert abs(u_sum - ref["U_sum"]) <= 1e-12 * uabs
        assert abs(u_mean - ref["U_mean"]) <= 1e-12 * uabs / uo.falling_factorial(9, 6)
        assert np.allclose(V, ref["V"], rtol=1e-13, atol=0)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("name,n,N", [("k4_cycle_rbf", 72, 3), ("path5_chord_linear_tanh", 200, 2),
                                      ("c4_rbf", 300, 2), ("triangle_rbf", 200, 3)])
def test_shards_on_one_gpu_sum_to_the_full_result(us, name, n, N, prec):
    import torch
    from paper_2508_12627_gb300.engine import Engine
    w = synth.workload(name, n)
    full = Engine(w.graph, w.factors, precision=prec).evaluate(w.X)
    tot = None
    for r in range(N):
        eng = Engine(w.graph, w.factors, precision=prec, shard=(r, N, n))
        out = eng.evaluate(w.X)
        V = out["V"]
        ev = np.array(eng.plan.info["evaluated"], dtype=bool)
        assert np.all(V[~ev] == 0.0)                              # other shards' partitions report 0
        vec = np.concatenate([[out["U_sum"], out["U_mean"]], V])
        tot = vec if tot is None else tot + vec
    torch.cuda.synchronize()
    a = uo.ustat(w.graph, w.factors, w.X, absolute=True)
    Vabs = np.maximum(np.array(a["V"]), 1e-300)
    uabs = float(np.abs(np.array(a["mu"], dtype=float)) @ np.array(a["V"]))
    # the parity tests' bounds at these sizes: float64 to 1e-11; split BF16 with
    # float32 storage below the full sample size to 5e-7 (1e-6 on the
    # heavy-tailed path + chord data)
    tol = 1e-11 if prec == "fp64" else (1e-6 if name == "path5_chord_linear_tanh" else 5e-7)
    assert np.all(np.abs(tot[2:] - full["V"]) <= tol * Vabs)
    assert abs(tot[0] - full["U_sum"]) <= tol * uabs
    ref = uo.ustat(w.graph, w.factors, w.X)
    assert abs(tot[0] - ref["U_sum"]) <= tol * uabs


def test_order_seven_chain_shards_cover_once_and_plan_quickly(us):
    # m = 7 (877 partitions): the estimates lower along the full plan's orders
    import time

    from paper_2508_12627_gb300 import hoif
    g, names = hoif.chain_graph(7)
    t0 = time.time()
    plans = [us.Plan(g, [us.MATRIX] * len(names), shard=(r, 2, 10000)) for r in range(2)]
    assert time.time() - t0 < 60.0
    owner = plans[0].owner
    assert plans[1].owner == owner and set(owner) == {0, 1}
    for r, p in enumerate(plans):
        assert p.info["evaluated"] == [int(o == r) for o in owner]
    full = us.Plan(g, [us.MATRIX] * len(names))
    f = [p.flops(10000)[0] for p in plans]
    assert max(f) <= 1.2 * full.flops(10000)[0] / 2


# ---------------------------------------------------------------- row shards of one evaluation
# (ustat_eval_rows / ustat_combine): each rank computes a contiguous range of the
# tiles of every n^3 product that feeds only reductions and of the values of every
# treewidth-3 step's eliminated index, the rest whole; the ranks' scalar arrays sum
# to the whole evaluation's scalars.

@pytest.mark.gpu
@pytest.mark.parametrize("name,n,N,prec", [("c4_rbf", 1100, 2, "bf16x3"), ("c4_rbf", 1100, 3, "bf16x3"),
                                           ("k4_cycle_rbf", 300, 2, "bf16x3"), ("k4_cycle_rbf", 300, 4, "bf16x4"),
                                           ("path5_chord_linear_tanh", 300, 3, "bf16x4"),
                                           ("triangle_rbf", 200, 2, "fp64")])
def test_row_shards_on_one_gpu_sum_to_the_whole_evaluation(us, name, n, N, prec):
    import torch
    from paper_2508_12627_gb300.engine import Engine
    w = synth.workload(name, n)
    eng = Engine(w.graph, w.factors, precision=prec)
    whole = eng.evaluate(w.X)
    parts = [eng.scalars_rows(w.X, r, N) for r in range(N)]
    torch.cuda.synchronize()
    one = eng.scalars_rows(w.X, 0, 1)
    tot = torch.stack(parts).sum(0)
    got = eng.combine(tot, n)
    a = uo.ustat(w.graph, w.factors, w.X, absolute=True)
    Vabs = np.maximum(np.array(a["V"]), 1e-300)
    # the same products in another grouping of the float64 atomic sums: agreement
    # far below the modes' tolerances
    assert np.all(np.abs(got["V"] - whole["V"]) <= 1e-12 * Vabs)
    assert np.allclose(one.cpu().numpy(), tot.cpu().numpy(), rtol=1e-12, atol=1e-300)
    ref = uo.ustat(w.graph, w.factors, w.X)
    tol = {"fp64": 1e-11, "bf16x3": 5e-7, "bf16x4": 1e-8}[prec]
    assert np.all(np.abs(got["V"] - np.array(ref["V"])) <= tol * Vabs)
    if prec == "fp64":
        # the CUDA-core products are not divided: rank 0 computes everything (the
        # same sums, up to the order of their float64 atomic additions)
        assert np.allclose(parts[0].cpu().numpy(), one.cpu().numpy(), rtol=1e-13, atol=0.0)
        assert all(not p.cpu().numpy().any() for p in parts[1:])
    else:
        # every rank has work in the sharded steps: no rank's array equals the whole
        for p in parts:
            assert not np.allclose(p.cpu().numpy(), one.cpu().numpy())


def _row_rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    from paper_2508_12627_gb300.engine import Engine
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # a stand-in for a rank's scalar array (no GPU here): rank r holds the r-th
    # term of a split of known values; the exchange must return their sum
    full = np.linspace(-3.0, 7.0, 41) ** 3
    noise = np.random.default_rng(7).standard_normal(41)
    mine = torch.as_tensor(full / 2 + (noise if rank == 0 else -noise))
    res = Engine.reduce_row_scalars(mine.clone())
    dist.destroy_process_group()
    q.put((rank, res.numpy().tolist()))


def test_two_gloo_ranks_sum_their_row_scalars():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_row_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    full = np.linspace(-3.0, 7.0, 41) ** 3
    for _, v in res:
        assert np.allclose(v, full, rtol=1e-14, atol=1e-12)


def test_row_shard_scalar_count_and_arguments(us):
    w = synth.workload("k4_cycle_rbf", 64)
    p = us.Plan(w.graph, [f.kind for f in w.factors], precision="bf16x3")
    assert us.scalar_count(p) > 0
    for rank, N in [(2, 2), (-1, 2), (0, 0)]:
        with pytest.raises(us.UstatError):
            us.ustat_eval_rows(p, rank, N, 256, 0, 64, 32, [(uo.RBF, 64.0, 0)], 256, 1 << 30, None, 256)
