"""The learned order ranker: its CUDA forward / backward / Adam kernels against
the FP64 oracle of the network, a training run, learned plans that give the
same U as the exhaustive planner's, and (on the stored held-out instances of
the committed weights) the regret the network saves over the flop-count pick."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import mlp_oracle as mo
from oracle import ustat_oracle as uo

F, H = 16, 32


@pytest.fixture(scope="module")
def us():
    from paper_2508_12627_gb300 import build
    build.build()
    from paper_2508_12627_gb300 import ustat
    return ustat


def _weights():
    from paper_2508_12627_gb300 import ranker
    if not os.path.exists(ranker.WEIGHTS):
        pytest.skip("no trained weights")
    return ranker.load()


def _rand(seed, rows=777):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, mo.param_count(F, H))
    X = rng.uniform(0, 1, (rows, F))
    t = rng.normal(0, 1, rows)
    return p.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64), t.astype(np.float32)


def test_candidates_and_contraction_plans(us):
    g = synth.path5_chord_graph()
    kinds = [uo.LINEAR, uo.TANH_DOT]
    orders, feats = us.order_candidates(g, kinds, 1024)
    assert len(orders) == len({tuple(o) for o in orders}) > 1
    assert all(sorted(o) == list(range(5)) for o in orders)
    assert all(len(f) == us.RANK_FEATURES for f in feats)
    assert all(abs(f[0] - 10 / 12) < 1e-6 for f in feats)          # log2 n / 12
    po = us.plan_orders(us.plan_contraction(g, kinds, None))[-1]
    assert us.order_features(g, kinds, 1024, po) in feats           # the planner's choice is a candidate
    p = us.plan_contraction(g, kinds, orders[0])
    ev = p.info["evaluated"]
    assert sum(ev) == 1 and ev[-1] == 1                              # only the finest partition
    with pytest.raises(us.UstatError):
        us.plan_contraction(g, kinds, [0, 0, 1, 2, 3])


@pytest.mark.gpu
def test_mlp_kernels_match_oracle(us):
    import torch
    p, X, t = _rand(0)
    st = torch.cuda.current_stream().cuda_stream
    dp = torch.as_tensor(p, dtype=torch.float32, device="cuda")
    dX = torch.as_tensor(X, dtype=torch.float32, device="cuda")
    dt = torch.as_tensor(t, dtype=torch.float32, device="cuda")
    y = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    us.mlp_forward(dp.data_ptr(), F, H, dX.data_ptr(), X.shape[0], y.data_ptr(), st)
    yr, _ = mo.forward(p, F, H, X)
    assert np.allclose(y.cpu().numpy(), yr, rtol=1e-5, atol=1e-5 * np.abs(yr).max())
    ws = torch.empty(us.mlp_workspace_bytes(F, H, X.shape[0]), dtype=torch.uint8, device="cuda")
    g = torch.empty_like(dp)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    us.mlp_loss_grad(dp.data_ptr(), F, H, dX.data_ptr(), dt.data_ptr(), X.shape[0], ws.data_ptr(), ws.numel(),
                     g.data_ptr(), loss.data_ptr(), st)
    lr_, gr = mo.loss_and_grad(p, F, H, X, t)
    assert abs(loss.item() - lr_) <= 1e-5 * lr_
    gg = g.cpu().numpy()
    assert np.all(np.abs(gg - gr) <= 1e-4 * np.abs(gr).max() + 1e-5 * np.abs(gr)), np.abs(gg - gr).max()
    # Adam, two steps
    m = torch.zeros_like(dp)
    v = torch.zeros_like(dp)
    pr, mr, vr = p.copy(), np.zeros_like(p), np.zeros_like(p)
    gfix = np.float32(gr).astype(np.float64)
    dg = torch.as_tensor(gfix, dtype=torch.float32, device="cuda")
    for step in (1, 2):
        us.mlp_adam(dp.data_ptr(), dg.data_ptr(), m.data_ptr(), v.data_ptr(), dp.numel(), 1e-2, 0.9, 0.999, 1e-8,
                    step, st)
        pr, mr, vr = mo.adam(pr, gfix, mr, vr, step, 1e-2, 0.9, 0.999, 1e-8)
    assert np.allclose(dp.cpu().numpy(), pr, rtol=0, atol=2e-6)


@pytest.mark.gpu
def test_training_reduces_the_loss(us):
    from paper_2508_12627_gb300 import ranker
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, (4000, us.RANK_FEATURES))
    y = np.log(1 + 5 * X[:, 1] * X[:, 10] + X[:, 3] ** 2)      # a smooth positive target
    net = ranker.MLP(seed=1)
    hist = net.train(X, y, steps=1500, lr=3e-3)
    assert hist[-1][1] < 0.05 * hist[0][1]
    pred = net.predict(X[:100])
    assert np.mean((pred - y[:100]) ** 2) < 0.05 * np.var(y)


@pytest.mark.gpu
@pytest.mark.parametrize("name,n", [("k4_cycle_rbf", 72), ("path5_chord_linear_tanh", 200), ("c4_rbf", 300)])
def test_learned_plans_give_the_same_U(us, name, n):
    import torch
    from paper_2508_12627_gb300 import engine, ranker
    wts = _weights()
    w = synth.workload(name, n)
    kinds = [f.kind for f in w.factors]
    params = torch.as_tensor(np.asarray(wts["params"], dtype=np.float32), device="cuda")
    ws = torch.empty(max(256, us.rank_workspace_bytes(w.graph, kinds)), dtype=torch.uint8, device="cuda")
    lp = us.plan_learned(w.graph, kinds, n, params.data_ptr(), wts["hidden"], ws.data_ptr(), ws.numel(),
                         torch.cuda.current_stream().cuda_stream, precision="fp64")
    eng = engine.Engine(w.graph, w.factors, precision="fp64")
    ref = eng.evaluate(w.X)
    eng.plan = lp
    out = eng.evaluate(w.X)
    a = uo.ustat(w.graph, w.factors, w.X, absolute=True)
    Vabs = np.maximum(np.array(a["V"]), 1e-300)
    assert np.all(np.abs(out["V"] - ref["V"]) <= 1e-11 * Vabs)
    uabs = float(np.abs(np.array(a["mu"], dtype=float)) @ np.array(a["V"]))
    assert abs(out["U_sum"] - ref["U_sum"]) <= 1e-11 * uabs


def test_network_beats_the_flop_count_pick_on_held_out_instances():
    # offline: the committed weights, the FP64 oracle of the network, and the
    # held-out instances measured when the weights were trained
    from paper_2508_12627_gb300 import ranker
    wts = _weights()
    p = np.asarray(wts["params"], dtype=np.float64)
    reg = ranker.regrets(wts["held_out"], lambda Fm: mo.forward(p, wts["features"], wts["hidden"], Fm)[0])
    assert len(wts["held_out"]) >= 50
    assert reg["learned"] < reg["analytic"]
    assert reg["learned"] <= reg["minfill"]


def test_checkpoint_and_record_files_round_trip(tmp_path):
    # host side only: the training state and the timing records survive a write
    # and a read unchanged
    from paper_2508_12627_gb300 import ranker
    rng = np.random.default_rng(1)
    p, m, v = (rng.normal(0, 1, 100).astype(np.float32) for _ in range(3))
    ranker.save_checkpoint(tmp_path / "c.npz", p, m, v, 1234)
    c = ranker.load_checkpoint(tmp_path / "c.npz")
    assert c["step"] == 1234 and all(np.array_equal(c[k], x) for k, x in (("params", p), ("m", m), ("v", v)))
    f = tmp_path / "recs.jsonl"
    assert ranker.read_records(f) == []
    recs = [{"n": 256, "ms": [0.5, 0.25], "features": [[0.1] * 20, [0.2] * 20]}, {"n": 512, "ms": [1.0]}]
    ranker.append_records(f, recs[:1])
    ranker.append_records(f, recs[1:])
    assert ranker.read_records(f) == recs
