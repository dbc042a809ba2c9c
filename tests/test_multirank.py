"""The multi-rank path of bench.py on CPU: world_size-2 gloo ranks.  Every rank
evaluates its own replica of the workload (weak scaling, no data-path
collective); the job's time is the slowest rank's and the value counts the
evaluations of all ranks.  The reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r "took" 10 (r + 1) ms for 4 steps
    t = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    dist.barrier()
    q.put((rank, t, bench.job_value(world, 4, t)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [r[1] for r in res] == [20.0, 20.0]
    assert res[0][2] == pytest.approx(2 * 4 / 0.020)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        workload, steps, warmup, gpus = "c4_rbf", 1, 1, 2

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A())
    assert buf.getvalue() == ""


@pytest.mark.parametrize("workload", ["c4_rbf", "triangle_rbf", "k4_cycle_rbf", "path5_chord_linear_tanh",
                                      "motifs4_er", "hoif_chain", "dcov_sectors", "batched"])
def test_reference_arm_bounded_sample_for_every_workload(monkeypatch, workload):
    # every workload's reference line with small time limits: one bounded sample
    # per step, scaled to the full step, the contract's keys
    sys.path.insert(0, ROOT)
    import json

    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(bench, "REFERENCE_STEP_S", 0.3)
    monkeypatch.setattr(bench, "REFERENCE_BUDGET_S", 1.0)

    class A:
        steps, warmup, gpus = 2, 1, 1

    A.workload = workload
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A())
    line = json.loads(buf.getvalue())
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "evals/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["higher_is_better"] is True
    assert line["ms_per_step"] >= line["sample_ms_per_step"] * 0.999


def test_sample_sizing_and_growth_exponents():
    sys.path.insert(0, ROOT)
    import bench
    import synth
    # the oracle's growth n^(M + 1) from the largest quotient treewidth M
    assert bench.max_treewidth(synth.cycle4_graph()) == 2
    assert bench.max_treewidth(synth.triangle_graph()) == 2
    assert bench.max_treewidth(synth.k4_plus_cycle_graph()) == 3
    assert bench.max_treewidth(synth.path5_chord_graph()) == 2
    # doubling stops before the predicted time passes the limit, and at the full size
    calls = []

    def fake(n):
        calls.append(n)
        return 1e-10 * n ** 3

    assert bench._sized(fake, 4096, 64, 3, 20.0) == (4096, 1e-10 * 4096 ** 3) and calls[-1] == 4096
    calls.clear()
    ns, t = bench._sized(fake, 10 ** 6, 64, 3, 20.0)
    assert ns == 4096 and t == 1e-10 * 4096 ** 3 and 1e-10 * 8192 ** 3 > 20.0
    assert calls == [64, 128, 256, 512, 1024, 2048, 4096]
