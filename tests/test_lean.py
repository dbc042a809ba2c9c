"""Memory-lean evaluation (ustat_eval_lean): no n x n factor or product stored,
the factor rows rebuilt from X in panels (the space discussion of Section 3.3's
remark on space complexity and of the appendix "A Discussion on the Space
Complexity").

CPU: the workspace sizes (the stored form beyond one GPU's memory at n = 147456,
the lean form a few percent of it), the plans and arguments it refuses, and the
closed form used at that size, pinned against the oracle.  GPU: the lean form
against the oracle with ragged panels, against the stored oracle values of the
4-cycle at n = 4096, against the stored form, and bit-exact against the closed
form at n = 147456, where the stored form does not fit.

The closed form: with the sample made of G groups of identical points, the
groups far apart, the RBF factor matrix is the group-equality indicator: 1
inside a group, and across groups at most exp(-128^2 / h), which is 0 in float32
for the bandwidths h = 2d used here and far below the rounding of every V_pi in
float64.  For a kernel graph whose every quotient is connected, each restricted
V-statistic then counts the index tuples with all blocks in one group:
V_pi = sum_g s_g^(blocks of pi), and U_sum = sum_g (s_g)_m, the ordered distinct
m-tuples inside one group.
"""
import math

import numpy as np
import pytest

import synth
from oracle import ustat_oracle as uo

N_BIG = 147456            # stored bf16x3 4-cycle workspace: about 304 GB
DEVICE_MIB = 284208       # one GB300's memory as nvidia-smi reports it


def groups_sample(n, G, d, seed):
    """n rows in G groups of identical points, the rows shuffled: group g sits at
    128 times the binary digits of g + 1 (coordinates 0 or 128, so every digit,
    norm and dot product is a small exact integer; two groups differ in at least
    one coordinate, a squared distance of at least 128^2).  Returns X and the
    group sizes."""
    assert (G + 1).bit_length() <= d
    rng = np.random.default_rng(seed)
    labels = rng.integers(0, G, n)
    X = np.zeros((n, d))
    for c in range((G + 1).bit_length()):
        X[:, c] = 128.0 * (((labels + 1) >> c) & 1)
    sizes = np.bincount(labels, minlength=G)
    return X, sizes


def closed_form(graph_m, rgs_list, sizes):
    V = [int(sum(int(s) ** (max(r) + 1) for s in sizes)) for r in rgs_list]
    U = int(sum(math.perm(int(s), graph_m) for s in sizes))
    return V, U


def _plan(us, name, prec="bf16x3"):
    w = synth.workload(name, n=300)
    return us.Plan(w.graph, [f.kind for f in w.factors], precision=prec)


@pytest.fixture(scope="module")
def us():
    pytest.importorskip("torch")
    from paper_2508_12627_gb300 import ustat
    return ustat


def test_lean_workspace_is_panel_sized(us):
    p = _plan(us, "c4_rbf")
    stored = p.workspace_bytes(N_BIG, 32)
    lean = us.lean_workspace_bytes(p, N_BIG, 32, 8192)
    assert stored > DEVICE_MIB * 2 ** 20          # the stored form does not fit one GPU
    assert lean < 0.08 * stored
    # linear in the panel height
    a, b = us.lean_workspace_bytes(p, N_BIG, 32, 4096), us.lean_workspace_bytes(p, N_BIG, 32, 8192)
    c = us.lean_workspace_bytes(p, N_BIG, 32, 16384)
    assert abs((c - b) - 2 * (b - a)) <= 4 * 1024 * 3


def test_lean_refuses_other_plans_and_arguments(us):
    for name, prec in [("path5_chord_linear_tanh", "bf16x3"), ("c4_rbf", "bf16x4"), ("c4_rbf", "fp64"),
                       ("k4_cycle_rbf", "bf16x3")]:
        with pytest.raises(us.UstatError) as e:
            us.lean_workspace_bytes(_plan(us, name, prec), 4096, 32, 1024)
        assert e.value.code == us.USTAT_ERR_UNSUPPORTED, (name, prec)
    p = _plan(us, "c4_rbf")
    for panel in (0, 100, 129):
        with pytest.raises(us.UstatError) as e:
            us.lean_workspace_bytes(p, 4096, 32, panel)
        assert e.value.code == us.USTAT_ERR_INVALID_ARG


@pytest.mark.parametrize("name", ["c4_rbf", "triangle_rbf"])
def test_closed_form_against_oracle(name):
    # the pin of the large-n expectation: the oracle on a small grouped sample
    w = synth.workload(name, n=40)
    X, sizes = groups_sample(40, 5, w.X.shape[1], seed=3)
    r = uo.ustat(w.graph, w.factors, X)
    V, U = closed_form(w.graph.m, r["rgs"], sizes)
    assert np.array_equal(np.asarray(r["V"]), np.asarray(V, dtype=float)), name
    assert r["U_sum"] == U


def test_closed_form_fails_a_planted_mistake():
    # blocks counted as vertices (s^m for every partition) breaks the pin
    w = synth.workload("c4_rbf", n=30)
    X, sizes = groups_sample(30, 4, w.X.shape[1], seed=5)
    r = uo.ustat(w.graph, w.factors, X)
    wrong = [int(sum(int(s) ** w.graph.m for s in sizes)) for _ in r["rgs"]]
    assert not np.array_equal(np.asarray(r["V"]), np.asarray(wrong, dtype=float))


# ---------------------------------------------------------------- GPU

@pytest.fixture(scope="module")
def eng_mod():
    import torch
    assert torch.cuda.is_available()
    from paper_2508_12627_gb300 import build
    build.build()
    from paper_2508_12627_gb300 import engine
    return engine


def _check(out, ref, absref, tol, label):
    Vabs = np.maximum(np.asarray(absref["V"]), 1e-300)
    err = np.abs(out["V"] - np.asarray(ref["V"])) / Vabs
    assert err.max() <= tol, (label, err.max(), int(err.argmax()))
    uabs = sum(abs(mu) * va for mu, va in zip(ref["mu"], absref["V"]))
    assert abs(out["U_sum"] - ref["U_sum"]) <= tol * uabs, label


@pytest.mark.gpu
@pytest.mark.parametrize("name,n,panel", [("c4_rbf", 300, 128), ("triangle_rbf", 200, 128), ("c4_rbf", 389, 256)])
def test_lean_against_oracle_and_stored_form(eng_mod, name, n, panel):
    # several panels with a ragged last one; the stored form on the same input
    w = synth.workload(name, n=n)
    ref, absref = uo.ustat(w.graph, w.factors, w.X), uo.ustat(w.graph, w.factors, w.X, absolute=True)
    eng = eng_mod.Engine(w.graph, w.factors, precision="bf16x3")
    lean = eng.evaluate_lean(w.X, panel_rows=panel)
    _check(lean, ref, absref, 5e-7, (name, n, "oracle"))
    stored = eng.evaluate(w.X)
    # the same digits and per-entry accumulation; the sums in another grouping (the
    # build's reductions add float32 partial sums of 32 entries, each rounded to
    # 2^-24 of its size, over other tiles: the stored form visits the upper
    # triangle and doubles it)
    _check(lean, {"V": stored["V"], "mu": ref["mu"], "U_sum": stored["U_sum"]}, absref, 1e-8, (name, n, "stored"))


@pytest.mark.gpu
def test_lean_c4_full_size_against_stored_oracle_values(eng_mod):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "workload_c4_rbf.json")) as f:
        g = json.load(f)
    w = synth.workload("c4_rbf")
    eng = eng_mod.Engine(w.graph, w.factors, precision="bf16x3")
    lean = eng.evaluate_lean(w.X, panel_rows=1024)
    _check(lean, {"V": g["V"], "mu": g["mu"], "U_sum": g["U_sum"]}, {"V": g["V_abs"]}, 1e-8, "c4 n=4096 lean")


@pytest.mark.gpu
@pytest.mark.parametrize("n,G,panel,lean_only", [(16384, 64, 4096, False), (N_BIG, 512, 8192, True)])
def test_lean_bit_exact_on_grouped_samples(eng_mod, n, G, panel, lean_only):
    # K is the exact group indicator: every V_pi and U_sum are integers below 2^53,
    # and every step of the bf16x3 path is exact on them
    w = synth.workload("c4_rbf", n=300)
    X, sizes = groups_sample(n, G, 32, seed=11)
    eng = eng_mod.Engine(w.graph, w.factors, precision="bf16x3")
    V, U = closed_form(w.graph.m, eng.plan.info["rgs"], sizes)
    assert max(V) < 2 ** 53
    lean = eng.evaluate_lean(X, panel_rows=panel)
    assert np.array_equal(lean["V"], np.asarray(V, dtype=float)), (n, np.abs(lean["V"] - V).max())
    assert lean["U_sum"] == float(U)
    if not lean_only:
        stored = eng.evaluate(X)
        assert np.array_equal(stored["V"], np.asarray(V, dtype=float))
