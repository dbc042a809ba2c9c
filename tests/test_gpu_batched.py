"""Batched evaluation (ustat_batched_*): many samples of uneven size on several
streams, eager and replayed from a captured CUDA graph, before and after
autotuning, against single-sample evaluation through ustat_eval and against the
FP64 oracle.  Plus the host-side schedule (no GPU needed)."""
import numpy as np
import pytest

import synth
from oracle import ustat_oracle as uo

# the batched path runs the same kernels as ustat_eval; only the order of
# floating-point atomic additions may differ (relative to V_abs)
SAME_PATH_TOL = 1e-12
SMALL_N_TOL = 5e-7   # float32 entries, at most 7 factors per term (as in the parity tests)


@pytest.fixture(scope="module")
def us():
    from paper_2508_12627_gb300 import build
    build.build()
    from paper_2508_12627_gb300 import ustat
    return ustat


def _graphs():
    return {"c4": synth.cycle4_graph(), "c5": synth.cycle(5)}


def test_schedule_balances_lanes(us):
    g = synth.cycle4_graph()
    p = us.Plan(g, [uo.RBF], precision="bf16x3")
    ns = synth.batched_sizes(64, 256, 4096, 0)
    b = us.Batched(p, ns, 16, max_lanes=4)
    lanes, lane_of = b.info()
    assert lanes == 4 and sorted(set(lane_of)) == [0, 1, 2, 3]
    # longest-processing-time: no lane carries more than the mean load plus the largest sample
    cost = [p.flops(n)[0] + 2e9 for n in ns]
    load = [sum(c for c, l in zip(cost, lane_of) if l == k) for k in range(4)]
    assert max(load) <= sum(cost) / 4 + max(cost)
    assert b.workspace_bytes() >= 4 * p.workspace_bytes(max(ns), 16)
    b.set_lanes(2)
    assert b.info()[0] == 2 and set(b.info()[1]) == {0, 1}
    with pytest.raises(us.UstatError):
        b.set_lanes(5)
    with pytest.raises(us.UstatError) as e:
        us.Batched(p, [3, 10], 16)
    assert e.value.code == us.USTAT_ERR_N_LT_M


def test_matrix_factors_are_rejected(us):
    g = synth.Graph(2, [(0, 1, 0)], [])
    p = us.Plan(g, [uo.MATRIX], precision="fp32")
    b = us.Batched(p, [4, 5], 1)
    with pytest.raises(us.UstatError) as e:
        b.run([256, 256], 0, [(uo.MATRIX, 0.0, 256)], 256, 1 << 30, None, 256, 256)
    assert e.value.code == us.USTAT_ERR_UNSUPPORTED


def _setup(us, name, prec, ns, d=16, max_lanes=4):
    import torch
    g = _graphs()[name]
    p = us.Plan(g, [uo.RBF], precision=prec)
    Xs = [synth.normal_X(n, d, 1000 + i) for i, n in enumerate(ns)]
    Xd = [torch.as_tensor(x, device="cuda:0") for x in Xs]
    b = us.Batched(p, ns, d, max_lanes=max_lanes)
    ws = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device="cuda:0")
    k = p.info["n_parts"]
    U = torch.full((len(ns), 2), float("nan"), dtype=torch.float64, device="cuda:0")
    V = torch.full((len(ns), k), float("nan"), dtype=torch.float64, device="cuda:0")
    facs = [(uo.RBF, 2.0 * d, 0)]
    return g, p, Xs, Xd, b, ws, U, V, facs


def _single(us, p, Xd, facs):
    import torch
    outs = []
    for x in Xd:
        n, d = x.shape
        ws = torch.empty(p.workspace_bytes(n, d), dtype=torch.uint8, device="cuda:0")
        o = torch.empty(2 + p.info["n_parts"], dtype=torch.float64, device="cuda:0")
        us.ustat_eval(p, x.data_ptr(), 0, n, d, facs, ws.data_ptr(), ws.numel(),
                      torch.cuda.current_stream().cuda_stream, o.data_ptr(), o.data_ptr() + 16)
        outs.append(o.cpu().numpy())
    return outs


def _check_same(U, V, singles, absV):
    U = U.cpu().numpy()
    V = V.cpu().numpy()
    for i, s in enumerate(singles):
        va = np.maximum(absV[i], 1e-300)
        assert np.all(np.abs(V[i] - s[2:]) <= SAME_PATH_TOL * va), i
        assert abs(U[i, 0] - s[0]) <= SAME_PATH_TOL * max(abs(s[0]), np.abs(va).sum())


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["c4", "c5"])
@pytest.mark.parametrize("prec", ["bf16x3", "fp64"])
def test_batched_matches_single_and_oracle(us, name, prec):
    import torch
    ns = [300, 5, 130, 40, 257, 64, 7, 129]
    g, p, Xs, Xd, b, ws, U, V, facs = _setup(us, name, prec, ns)
    st = torch.cuda.current_stream().cuda_stream
    xp = [x.data_ptr() for x in Xd]
    b.run(xp, 0, facs, ws.data_ptr(), ws.numel(), st, U.data_ptr(), V.data_ptr())
    torch.cuda.synchronize()
    singles = _single(us, p, Xd, facs)
    absV = []
    for i, X in enumerate(Xs):
        ref = uo.ustat(g, [synth.Factor(uo.RBF, 2.0 * X.shape[1], None)], X)
        ab = uo.ustat(g, [synth.Factor(uo.RBF, 2.0 * X.shape[1], None)], X, absolute=True)
        absV.append(np.array(ab["V"]))
        tol = 1e-11 if prec == "fp64" else SMALL_N_TOL
        Vb = V[i].cpu().numpy()
        assert np.all(np.abs(Vb - np.array(ref["V"])) <= tol * np.maximum(absV[-1], 1e-300)), (name, i)
    _check_same(U, V, singles, absV)

    # one captured graph, replayed twice, gives the eager results
    U2 = torch.full_like(U, float("nan"))
    V2 = torch.full_like(V, float("nan"))
    s2 = torch.cuda.Stream()
    with torch.cuda.stream(s2):
        b.capture(xp, 0, facs, ws.data_ptr(), ws.numel(), s2.cuda_stream, U2.data_ptr(), V2.data_ptr())
        for _ in range(2):
            V2.fill_(float("nan"))
            b.replay(s2.cuda_stream)
    torch.cuda.synchronize()
    _check_same(U2, V2, singles, absV)


@pytest.mark.gpu
def test_autotune_keeps_results(us):
    import torch
    ns = [700, 1100, 256, 2100, 300, 900]
    g, p, Xs, Xd, b, ws, U, V, facs = _setup(us, "c5", "bf16x3", ns)
    st = torch.cuda.current_stream().cuda_stream
    xp = [x.data_ptr() for x in Xd]
    b.run(xp, 0, facs, ws.data_ptr(), ws.numel(), st, U.data_ptr(), V.data_ptr())
    torch.cuda.synchronize()
    U0, V0 = U.clone(), V.clone()
    lanes, ms = b.autotune(xp, 0, facs, ws.data_ptr(), ws.numel(), st, U.data_ptr(), V.data_ptr())
    assert lanes in (1, 2, 4) and ms > 0
    U.fill_(float("nan"))
    V.fill_(float("nan"))
    b.run(xp, 0, facs, ws.data_ptr(), ws.numel(), st, U.data_ptr(), V.data_ptr())
    torch.cuda.synchronize()
    # another GEMM tile shape changes the summation order inside the tensor-core
    # accumulators: same 1e-8 target as every bf16x3 result
    v0, v1 = V0.cpu().numpy(), V.cpu().numpy()
    assert np.all(np.abs(v1 - v0) <= 1e-8 * np.abs(v0))


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["c4", "c5"])
def test_full_batch_against_stored_oracle_values(us, name):
    # the batched workload at its full size: all 512 samples (n uniform in
    # [256, 4096], d = 16) in one captured graph on 16 lanes, in the launch
    # configuration bench.py times; the samples whose values the oracle stored
    # (tests/golden/make_workload_golden.py: the smallest, the largest and six
    # more) match to 1e-8 of V_abs, and every sample's results are finite
    import json
    import os
    import torch
    with open(os.path.join(os.path.dirname(__file__), "golden", "workload_batched.json")) as f:
        gold = json.load(f)
    ns = [int(v) for v in synth.batched_sizes(512, 256, 4096, 0)]
    g, p, Xs, Xd, b, ws, U, V, facs = _setup(us, name, "bf16x3", ns, max_lanes=16)
    s2 = torch.cuda.Stream()
    xp = [x.data_ptr() for x in Xd]
    with torch.cuda.stream(s2):
        b.capture(xp, 0, facs, ws.data_ptr(), ws.numel(), s2.cuda_stream, U.data_ptr(), V.data_ptr())
        b.replay(s2.cuda_stream)
    torch.cuda.synchronize()
    Uh, Vh = U.cpu().numpy(), V.cpu().numpy()
    assert np.all(np.isfinite(Uh)) and np.all(np.isfinite(Vh))
    checked = 0
    for rec in gold["samples"]:
        if rec["graph"] != name:
            continue
        i = rec["index"]
        assert rec["n"] == ns[i]
        Vabs = np.array(rec["V_abs"])
        assert np.all(np.abs(Vh[i] - np.array(rec["V"])) <= 1e-8 * Vabs), (name, i)
        assert abs(Uh[i, 0] - rec["U_sum"]) <= 1e-8 * rec["U_abs"], (name, i)
        checked += 1
    assert checked == 8


def test_grouped_form_arguments(us):
    g = synth.cycle4_graph()
    p = us.Plan(g, [uo.RBF], precision="bf16x3")
    ns = [300, 700, 129]
    b = us.Batched(p, ns, 16, max_lanes=2)
    lane_bytes = b.workspace_bytes()
    b.set_grouped(True)
    # one region per sample, plus the group images
    assert b.workspace_bytes() >= sum(p.workspace_bytes(n, 16) for n in ns)
    b.set_grouped(False)
    assert b.workspace_bytes() == lane_bytes
    p64 = us.Plan(g, [uo.RBF], precision="fp64")
    with pytest.raises(us.UstatError) as e:
        us.Batched(p64, ns, 16).set_grouped(True)
    assert e.value.code == us.USTAT_ERR_UNSUPPORTED


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["c4", "c5"])
def test_grouped_form_matches_lanes_and_oracle(us, name):
    # every product step of all samples in one persistent launch: the same digits
    # and per-entry accumulation as the lane form, the reductions added in another
    # order; eager, and a captured graph replayed twice
    import torch
    ns = [300, 5, 130, 40, 257, 64, 7, 129, 1100, 700]
    g, p, Xs, Xd, b, ws, U, V, facs = _setup(us, name, "bf16x3", ns)
    st = torch.cuda.current_stream().cuda_stream
    xp = [x.data_ptr() for x in Xd]
    b.run(xp, 0, facs, ws.data_ptr(), ws.numel(), st, U.data_ptr(), V.data_ptr())
    torch.cuda.synchronize()
    U0, V0 = U.cpu().numpy(), V.cpu().numpy()
    b.set_grouped(True)
    wg = torch.full((b.workspace_bytes(),), 255, dtype=torch.uint8, device="cuda:0")
    U.fill_(float("nan"))
    V.fill_(float("nan"))
    b.run(xp, 0, facs, wg.data_ptr(), wg.numel(), st, U.data_ptr(), V.data_ptr())
    torch.cuda.synchronize()
    absV = []
    for i, X in enumerate(Xs):
        ab = uo.ustat(g, [synth.Factor(uo.RBF, 2.0 * X.shape[1], None)], X, absolute=True)
        absV.append(np.maximum(np.array(ab["V"]), 1e-300))
        assert np.all(np.abs(V[i].cpu().numpy() - V0[i]) <= SAME_PATH_TOL * absV[-1]), (name, i)
        assert abs(U[i, 0].item() - U0[i, 0]) <= SAME_PATH_TOL * absV[-1].sum(), (name, i)
        if ns[i] <= 300:
            ref = uo.ustat(g, [synth.Factor(uo.RBF, 2.0 * X.shape[1], None)], X)
            assert np.all(np.abs(V[i].cpu().numpy() - np.array(ref["V"])) <= SMALL_N_TOL * absV[-1]), (name, i)
    U2 = torch.full_like(U, float("nan"))
    V2 = torch.full_like(V, float("nan"))
    s2 = torch.cuda.Stream()
    with torch.cuda.stream(s2):
        b.capture(xp, 0, facs, wg.data_ptr(), wg.numel(), s2.cuda_stream, U2.data_ptr(), V2.data_ptr())
        for _ in range(2):
            V2.fill_(float("nan"))
            b.replay(s2.cuda_stream)
    torch.cuda.synchronize()
    for i in range(len(ns)):
        assert np.all(np.abs(V2[i].cpu().numpy() - V0[i]) <= SAME_PATH_TOL * absV[i]), (name, i)


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["c4", "c5"])
def test_full_batch_grouped_against_stored_oracle_values(us, name):
    # all 512 samples of the batched workload, every product step one launch over
    # all samples' tiles, captured and replayed: the stored oracle values to 1e-8
    import json
    import os
    import torch
    with open(os.path.join(os.path.dirname(__file__), "golden", "workload_batched.json")) as f:
        gold = json.load(f)
    ns = [int(v) for v in synth.batched_sizes(512, 256, 4096, 0)]
    g, p, Xs, Xd, b, ws, U, V, facs = _setup(us, name, "bf16x3", ns, max_lanes=16)
    del ws
    b.set_grouped(True)
    wg = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device="cuda:0")
    s2 = torch.cuda.Stream()
    xp = [x.data_ptr() for x in Xd]
    with torch.cuda.stream(s2):
        b.capture(xp, 0, facs, wg.data_ptr(), wg.numel(), s2.cuda_stream, U.data_ptr(), V.data_ptr())
        b.replay(s2.cuda_stream)
    torch.cuda.synchronize()
    Uh, Vh = U.cpu().numpy(), V.cpu().numpy()
    assert np.all(np.isfinite(Uh)) and np.all(np.isfinite(Vh))
    checked = 0
    for rec in gold["samples"]:
        if rec["graph"] != name:
            continue
        i = rec["index"]
        Vabs = np.array(rec["V_abs"])
        assert np.all(np.abs(Vh[i] - np.array(rec["V"])) <= 1e-8 * Vabs), (name, i)
        assert abs(Uh[i, 0] - rec["U_sum"]) <= 1e-8 * rec["U_abs"], (name, i)
        checked += 1
    assert checked == 8
