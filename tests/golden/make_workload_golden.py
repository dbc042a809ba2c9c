"""Write the stored expected values of the five workloads at their full sizes.

Calls only the FP64 oracle (oracle/ustat_oracle.py) on the seeded inputs of the
``synth`` module; nothing here touches the CUDA library.  For every workload it
stores, per partition pi of [m] in restricted-growth-string order, mu_pi and the
restricted V-statistic V_pi (Definition "Restricted V-Statistic", Section 3.3), the
same contraction on the entrywise absolute values of the factors (V_abs, the scale
against which the rounding of a sum with cancellation is judged), and U_sum =
sum_pi mu_pi V_pi, U_mean = U_sum / (n)_m (Lemma "Decomposition of U-Statistic into
V-Statistics").  Where every factor entry is positive (the RBF kernel) V_abs = V
and the absolute pass is not repeated.

Usage:  python tests/golden/make_workload_golden.py [name ...]
names:  triangle_rbf c4_rbf path5_chord_linear_tanh k4_cycle_rbf batched
The full set takes about an hour on eight cores (the path + chord workload at
n = 16384 and K4 + cycle at n = 1024 dominate).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import ustat_oracle as uo  # noqa: E402

# sample indices of the 512-sample batched workload stored here: the smallest and
# the largest n, and six more spread over the index range
BATCHED_PICK = 8


def _positive(graph, factors, X) -> bool:
    return all(f.kind == uo.RBF for f in factors)


def evaluate(graph, factors, X) -> dict:
    t0 = time.time()
    r = uo.ustat(graph, factors, X)
    if _positive(graph, factors, X):
        vabs = list(r["V"])
    else:
        vabs = uo.ustat(graph, factors, X, absolute=True)["V"]
    uabs = float(sum(abs(mu) * v for mu, v in zip(r["mu"], vabs)))
    return {"n": int(X.shape[0]), "d": int(X.shape[1]), "m": graph.m,
            "rgs": [list(p) for p in r["rgs"]], "mu": [int(x) for x in r["mu"]],
            "V": [float(v) for v in r["V"]], "V_abs": [float(v) for v in vabs],
            "U_sum": float(r["U_sum"]), "U_mean": float(r["U_mean"]), "U_abs": uabs,
            "oracle_seconds": round(time.time() - t0, 1)}


def batched_pick(sizes) -> list[int]:
    idx = {int(np.argmin(sizes)), int(np.argmax(sizes))}
    for k in np.linspace(0, len(sizes) - 1, BATCHED_PICK - 2 + 2).astype(int)[1:-1]:
        idx.add(int(k))
    return sorted(idx)


def main(names):
    for name in names:
        if name == "batched":
            samples = synth.batched_workload()
            sizes = np.array([n for n, _ in samples])
            out = {"workload": "batched", "d": 16, "samples": []}
            for i in batched_pick(sizes):
                n, X = samples[i]
                for gname, g in (("c4", synth.cycle4_graph()), ("c5", synth.cycle(5))):
                    rec = evaluate(g, [synth.rbf(16)], X)
                    rec.update({"index": i, "graph": gname})
                    out["samples"].append(rec)
                    print(name, i, n, gname, rec["oracle_seconds"], "s", flush=True)
        else:
            w = synth.workload(name)
            out = evaluate(w.graph, w.factors, w.X)
            out["workload"] = name
            print(name, w.n, out["oracle_seconds"], "s", flush=True)
        out["source"] = ("oracle/ustat_oracle.py (FP64 partition sum) on synth's seeded inputs, "
                         "written by tests/golden/make_workload_golden.py")
        with open(os.path.join(HERE, "workload_%s.json" % name), "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or ["triangle_rbf", "c4_rbf", "batched", "k4_cycle_rbf", "path5_chord_linear_tanh"])
