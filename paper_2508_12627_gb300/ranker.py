"""Learned elimination-order ranker: training data from measured times of the
planner's own candidate orders, training with the library's MLP kernels
(forward, backward, Adam on the GPU), regret evaluation, and the weights file.

    python -m paper_2508_12627_gb300.ranker --graphs 5000 --out <weights.json>

Each instance is a random connected kernel graph G(m, p) (m in 3..7, p in
[0.3, 0.8], up to two unary factors) at a sample size n.  For the graph's own
contraction (every vertex a distinct index) the instance measures the
evaluation time (CUDA events, median of two after a warm-up) of a few of its distinct elimination sequences
(ustat_order_candidates) and of the plans the exhaustive and min-fill planners
pick.  The network learns log(time) from a sequence's features; the planner
then picks per partition the candidate of least predicted time
(ustat_plan_learned).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import ustat as us

HIDDEN = 32
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ranker_weights.json")
RBF, TANH = us.RBF, us.TANH_DOT
KINDS = [RBF, TANH]


def random_graph(rng):
    import synth
    m = int(rng.integers(3, 8))
    p = float(rng.uniform(0.3, 0.8))
    return synth.random_connected_graph(rng, m, p, max_unary=2)


def sample_size(rng, tw):
    """n for an instance: up to 2048, up to 512 when an n^4 step is needed."""
    return int(rng.choice([128, 256, 384, 512] if tw >= 3 else [256, 512, 1024, 2048]))


def graph_dict(g):
    return {"m": g.m, "edges": [list(e) for e in g.edges], "unary": [list(u) for u in g.unary]}


class Timer:
    """Evaluates plans on one device buffer set and times them with CUDA events."""

    def __init__(self, d=16, ws_bytes=1 << 31, seed=7):
        import torch
        self.torch = torch
        self.d = d
        self.ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
        rng = np.random.default_rng(seed)
        self.w = torch.as_tensor(rng.normal(0, 1 / math.sqrt(d), d), device="cuda")
        self.X = {}
        self.out = torch.empty(2 + 877, dtype=torch.float64, device="cuda")
        self.stream = torch.cuda.current_stream()

    def x(self, n):
        if n not in self.X:
            import synth
            self.X[n] = self.torch.as_tensor(synth.normal_X(n, self.d, 11), device="cuda")
        return self.X[n]

    def factors(self):
        return [(RBF, 2.0 * self.d, 0), (TANH, 0.0, self.w.data_ptr())]

    def run(self, plan, n):
        X = self.x(n)
        need = plan.workspace_bytes(n, self.d)
        if need > self.ws.numel():
            raise MemoryError("workspace")
        us.ustat_eval(plan, X.data_ptr(), 0, n, self.d, self.factors(), self.ws.data_ptr(), self.ws.numel(),
                      self.stream.cuda_stream, self.out.data_ptr(), self.out.data_ptr() + 16)

    def time(self, plan, n, reps=2):
        torch = self.torch
        self.run(plan, n)
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            self.run(plan, n)
            b.record(self.stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))


def measure_instance(timer, g, rng, max_cand=5):
    """Times of a few distinct elimination sequences of the graph's contraction,
    and of the sequences the exhaustive and min-fill planners choose (these
    two are also candidates, with their features)."""
    base = {name: us.plan_contraction(g, KINDS, None, planner=pl)
            for name, pl in (("exhaustive", us.PLAN_EXHAUSTIVE), ("minfill", us.PLAN_MINFILL))}
    n = sample_size(rng, base["exhaustive"].info["tw"][-1])
    orders, feats = us.order_candidates(g, KINDS, n)
    if not orders:
        return None
    pick = list(range(len(orders)))
    if len(pick) > max_cand:
        pick = sorted(rng.choice(len(orders), max_cand, replace=False).tolist())
    rec = {"graph": graph_dict(g), "n": n, "features": [], "ms": [], "order": [], "candidates": len(orders)}
    for i in pick:
        p = us.plan_contraction(g, KINDS, orders[i])
        rec["features"].append(feats[i])
        rec["order"].append(orders[i])
        rec["ms"].append(timer.time(p, n))
    for name, p in base.items():
        order = [v for v in us.plan_orders(p)[-1] if v >= 0]
        t = timer.time(p, n)
        rec[name + "_ms"] = t
        rec["features"].append(us.order_features(g, KINDS, n, order))
        rec["order"].append(order)
        rec["ms"].append(t)
    return rec


def generate(count, seed, budget_s, timer=None, log=None, on_record=None):
    """Up to ``count`` measured instances within ``budget_s``; ``on_record`` (if
    given) receives each record as soon as it is measured."""
    timer = timer or Timer()
    rng = np.random.default_rng(seed)
    recs = []
    t0 = time.time()
    while len(recs) < count and time.time() - t0 < budget_s:
        g = random_graph(rng)
        try:
            r = measure_instance(timer, g, rng)
        except us.UstatError as e:
            if e.code in (us.USTAT_ERR_TW_TOO_LARGE, us.USTAT_ERR_UNSUPPORTED):
                continue
            raise
        if r is not None:
            recs.append(r)
            if on_record:
                on_record(r)
        if log and len(recs) % 250 == 0:
            log("%d instances, %.0f s" % (len(recs), time.time() - t0))
    return recs


class MLP:
    """The ranker network on the GPU (parameters, Adam state) driven through the
    library's MLP kernels."""

    def __init__(self, hidden=HIDDEN, seed=0, params=None):
        import torch
        self.torch = torch
        self.F = us.RANK_FEATURES
        self.H = hidden
        self.P = us.mlp_param_count(self.F, self.H)
        if params is None:
            rng = np.random.default_rng(seed)
            W1 = rng.normal(0, math.sqrt(2.0 / self.F), (self.H, self.F))
            W2 = rng.normal(0, math.sqrt(2.0 / self.H), (self.H, self.H))
            w3 = rng.normal(0, math.sqrt(1.0 / self.H), self.H)
            params = np.concatenate([W1.ravel(), np.zeros(self.H), W2.ravel(), np.zeros(self.H), w3, [0.0]])
        self.params = torch.as_tensor(np.asarray(params, dtype=np.float32), device="cuda").contiguous()
        assert self.params.numel() == self.P
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.step_no = 0

    def predict(self, feats):
        torch = self.torch
        X = torch.as_tensor(np.asarray(feats, dtype=np.float32), device="cuda").contiguous()
        y = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
        us.mlp_forward(self.params.data_ptr(), self.F, self.H, X.data_ptr(), X.shape[0], y.data_ptr(),
                       torch.cuda.current_stream().cuda_stream)
        return y.cpu().numpy()

    def train(self, feats, targets, steps=4000, lr=2e-3, log=None):
        torch = self.torch
        X = torch.as_tensor(np.asarray(feats, dtype=np.float32), device="cuda").contiguous()
        t = torch.as_tensor(np.asarray(targets, dtype=np.float32), device="cuda").contiguous()
        rows = X.shape[0]
        ws = torch.empty(us.mlp_workspace_bytes(self.F, self.H, rows), dtype=torch.uint8, device="cuda")
        st = torch.cuda.current_stream().cuda_stream
        hist = []
        for k in range(steps):
            # cosine decay of the step size
            lr_k = lr * 0.5 * (1 + math.cos(math.pi * k / steps))
            us.mlp_loss_grad(self.params.data_ptr(), self.F, self.H, X.data_ptr(), t.data_ptr(), rows,
                             ws.data_ptr(), ws.numel(), self.grad.data_ptr(), self.loss.data_ptr(), st)
            self.step_no += 1
            us.mlp_adam(self.params.data_ptr(), self.grad.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.P,
                        lr_k, 0.9, 0.999, 1e-8, self.step_no, st)
            if k % 500 == 0 or k == steps - 1:
                hist.append((k, float(self.loss.item())))
                if log:
                    log("step %d loss %.5f" % hist[-1])
        return hist

    def numpy(self):
        return self.params.cpu().numpy().astype(np.float64)

    def save(self, path):
        """Checkpoint: parameters, Adam moments and step count."""
        save_checkpoint(path, self.params.cpu().numpy(), self.m.cpu().numpy(), self.v.cpu().numpy(), self.step_no)

    @classmethod
    def restore(cls, path, hidden=HIDDEN):
        """A network in the state save() wrote; train() continues from it."""
        c = load_checkpoint(path)
        net = cls(hidden=hidden, params=c["params"])
        net.m.copy_(net.torch.from_numpy(c["m"]))
        net.v.copy_(net.torch.from_numpy(c["v"]))
        net.step_no = c["step"]
        return net


def save_checkpoint(path, params, m, v, step):
    """The network's training state: parameters, Adam moments and step count
    (float32 arrays as trained, written without rounding)."""
    np.savez(path, params=np.asarray(params, dtype=np.float32), m=np.asarray(m, dtype=np.float32),
             v=np.asarray(v, dtype=np.float32), step=np.int64(step))


def load_checkpoint(path):
    with np.load(path) as z:
        return {"params": z["params"].copy(), "m": z["m"].copy(), "v": z["v"].copy(), "step": int(z["step"])}


def append_records(path, recs):
    """Timing records, one JSON object per line, appended: an interrupted data
    generation keeps what it measured."""
    with open(path, "a") as f:
        for r in recs:
            f.write(json.dumps(r) + "\n")


def read_records(path):
    if not os.path.exists(path):
        return []
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]


def regrets(recs, score):
    """Per instance: the measured candidate the scorer picks, its time over the
    best measured time (candidates and the two planners' plans) minus 1."""
    out = {"learned": [], "analytic": [], "exhaustive": [], "minfill": []}
    for r in recs:
        ms = np.array(r["ms"])
        best = min(ms.min(), r["exhaustive_ms"], r["minfill_ms"])
        s = score(np.array(r["features"], dtype=np.float64))
        out["learned"].append(ms[int(np.argmin(s))] / best - 1)
        # the flop-count pick (total flops, then n^4, n^3 and step counts)
        f = np.array(r["features"])
        key = [tuple(np.round(row[[10, 12, 11]], 6)) + (row[1:10].sum(),) for row in f]
        out["analytic"].append(ms[min(range(len(key)), key=lambda i: key[i])] / best - 1)
        out["exhaustive"].append(r["exhaustive_ms"] / best - 1)
        out["minfill"].append(r["minfill_ms"] / best - 1)
    return {k: float(np.mean(v)) for k, v in out.items()}


def compare_plans(cases, wts, reps=5, log=None):
    """Whole plans (all partitions, with the sharing between them) chosen by the
    exhaustive, min-fill and learned planners, timed on the same inputs: per case
    {name, m, n, partitions, ms: {planner: ms}, flops: {planner: plan flops},
    max_rel_diff: the learned plan's largest V difference from the exhaustive
    plan's, relative to |V|}.  A case is (name, graph, factors, kinds, X, precision)
    with factors as ustat_eval takes them (device data)."""
    import torch
    params = torch.as_tensor(np.asarray(wts["params"], dtype=np.float32), device="cuda")
    st = torch.cuda.current_stream()
    out = []
    for name, g, facs, kinds, X, prec in cases:
        n, d = X.shape
        rws = torch.empty(max(256, us.rank_workspace_bytes(g, kinds, prec)), dtype=torch.uint8, device="cuda")
        plans = {"exhaustive": us.Plan(g, kinds, precision=prec, planner=us.PLAN_EXHAUSTIVE),
                 "minfill": us.Plan(g, kinds, precision=prec, planner=us.PLAN_MINFILL),
                 "learned": us.plan_learned(g, kinds, n, params.data_ptr(), wts["hidden"], rws.data_ptr(),
                                            rws.numel(), st.cuda_stream, precision=prec)}
        need = max(p.workspace_bytes(n, d) for p in plans.values())
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        res = {"name": name, "m": g.m, "n": int(n), "partitions": plans["exhaustive"].info["n_parts"], "ms": {},
               "flops": {}}
        V = {}
        for pn, p in plans.items():
            o = torch.empty(2 + p.info["n_parts"], dtype=torch.float64, device="cuda")

            def run():
                us.ustat_eval(p, X.data_ptr(), 0 if X.dtype == torch.float64 else 1, n, d, facs, ws.data_ptr(),
                              ws.numel(), st.cuda_stream, o.data_ptr(), o.data_ptr() + 16)
            run()
            ts = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                run()
                b.record(st)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            res["ms"][pn] = float(np.median(ts))
            res["flops"][pn] = float(p.flops(n)[0])
            V[pn] = o[2:].cpu().numpy()
        res["max_rel_diff"] = float(np.max(np.abs(V["learned"] - V["exhaustive"]) /
                                           np.maximum(np.abs(V["exhaustive"]), 1e-300)))
        if log:
            log(json.dumps(res))
        out.append(res)
        del ws
    return out


def comparison_cases(count=20, seed=31):
    """Configurations 5 (K4 + cycle, n = 1024) and 3 (path + chord, n = 16384) and
    `count` random connected kernel graphs G(m, p), m = 6 or 7, p in [0.15, 0.55] (RBF edges, up
    to two tanh unary factors) at n = 2048, or 512 when a partition needs an n^4
    step."""
    import torch
    import synth
    cases = []
    for wname in ("k4_cycle_rbf", "path5_chord_linear_tanh"):
        w = synth.workload(wname)
        X = torch.as_tensor(np.ascontiguousarray(w.X), device="cuda")
        keep = []
        facs = []
        for f in w.factors:
            if f.data is not None:
                t = torch.as_tensor(np.ascontiguousarray(f.data, dtype=np.float64), device="cuda")
                keep.append(t)
                facs.append((f.kind, f.param, t.data_ptr()))
            else:
                facs.append((f.kind, f.param, 0))
        cases.append((wname, w.graph, facs, [f.kind for f in w.factors], X, "bf16x3"))
        cases[-1] = cases[-1] + (keep,)
    rng = np.random.default_rng(seed)
    d = 16
    w = torch.as_tensor(rng.normal(0, 1 / math.sqrt(d), d), device="cuda")
    while len(cases) < count + 2:
        m = int(rng.integers(6, 8))
        g = synth.random_connected_graph(rng, m, float(rng.uniform(0.15, 0.55)), max_unary=2)
        try:
            p = us.Plan(g, KINDS, precision="bf16x3")
        except us.UstatError:   # treewidth above 3
            continue
        if p.info["n_parts"] < 2:
            continue
        n = 512 if max(p.info["tw"]) >= 3 else 2048
        X = torch.as_tensor(synth.normal_X(n, d, 100 + len(cases)), device="cuda")
        cases.append(("random m=%d tw=%d" % (m, max(p.info["tw"])), g, [(RBF, 2.0 * d, 0), (TANH, 0.0, w.data_ptr())],
                      KINDS, X, "bf16x3", [w]))
    return [c[:6] for c in cases], [c[6] for c in cases]


def load(path=WEIGHTS):
    with open(path) as f:
        return json.load(f)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=5000)
    ap.add_argument("--budget", type=float, default=900.0, help="seconds for data generation")
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--data", default=None,
                    help="JSONL file of timing records: the records already in it are used, new ones are appended "
                         "as they are measured (an interrupted run resumes)")
    ap.add_argument("--checkpoint", default=None, help="write the trained network's state (npz) here")
    ap.add_argument("--compare-plans", default=None, metavar="OUT",
                    help="time whole plans of the exhaustive, min-fill and learned planners on configurations 5 "
                         "and 3 and 20 random m = 6-7 graphs, write the results (JSON) to OUT and stop")
    args = ap.parse_args()
    import torch
    from . import build
    build.build()
    torch.cuda.init()

    def log(s):
        print(s, flush=True)

    if args.compare_plans:
        cases, keep = comparison_cases()
        res = compare_plans(cases, load(), log=log)
        with open(args.compare_plans, "w") as f:
            json.dump(res, f, indent=1)
        del keep
        return

    timer = Timer()
    recs = read_records(args.data) if args.data else []
    if len(recs) < args.graphs:
        # a resumed run draws its graphs from a seed offset by the records it has
        recs += generate(args.graphs - len(recs), args.seed + len(recs), args.budget, timer, log,
                         on_record=(lambda r: append_records(args.data, [r])) if args.data else None)
    rng = np.random.default_rng(args.seed + 1)
    idx = rng.permutation(len(recs))
    n_test = max(1, len(recs) // 5)
    test = [recs[i] for i in idx[:n_test]]
    train = [recs[i] for i in idx[n_test:]]
    X = [f for r in train for f in r["features"]]
    y = [math.log(t) for r in train for t in r["ms"]]
    net = MLP()
    hist = net.train(X, y, steps=args.steps, log=log)
    if args.checkpoint:
        net.save(args.checkpoint)
    params = net.numpy()
    reg = regrets(test, lambda F: net.predict(F))
    log("held-out regret %s" % json.dumps(reg))
    # held-out instances in compact form, for the offline gain check
    held = [{"n": r["n"], "features": r["features"], "ms": r["ms"], "exhaustive_ms": r["exhaustive_ms"],
             "minfill_ms": r["minfill_ms"]} for r in test]
    out = {"features": us.RANK_FEATURES, "hidden": HIDDEN, "params": [float(v) for v in params],
           "instances": len(recs), "train_rows": len(X), "loss_history": hist, "held_out_regret": reg,
           "held_out": held, "generator": {"seed": args.seed, "graphs_requested": args.graphs,
                                           "budget_s": args.budget}}
    with open(args.out, "w") as f:
        json.dump(out, f)
    log("wrote %s (%d instances, %d rows)" % (args.out, len(recs), len(X)))


if __name__ == "__main__":
    main()
