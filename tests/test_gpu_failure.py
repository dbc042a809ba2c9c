"""GPU tests of the failure paths: a bounded device wait that runs out, and
non-finite inputs.  Nothing here faults or hangs the GPU: the wait runs out
because a test hook (ustat_debug_set_wait, off by default) shortens the wait
limit and makes the GEMM's copy warp issue no copy, so its MMA warp's first wait
gives up with nothing in flight; every kernel then returns and the host reads
the error word through ustat_status."""
import numpy as np
import pytest

import synth
from oracle import ustat_oracle as uo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_2508_12627_gb300 import build
    build.build()
    from paper_2508_12627_gb300 import engine
    from paper_2508_12627_gb300 import ustat as us
    return torch, engine, us


def _status(torch, us, eng):
    return us.status(eng._ws.data_ptr(), torch.cuda.current_stream().cuda_stream)


def _close(out, ref, tol):
    scale = max(abs(v) for v in ref["V"])
    assert np.all(np.abs(out["V"] - np.array(ref["V"])) <= tol * scale)


@pytest.mark.parametrize("name,n,prec", [("c4_rbf", 300, "bf16x3"), ("k4_cycle_rbf", 72, "bf16x3"),
                                         ("path5_chord_linear_tanh", 257, "bf16x4")])
def test_bounded_wait_runs_out_then_recovers(env, name, n, prec):
    torch, engine, us = env
    w = synth.workload(name, n)
    eng = engine.Engine(w.graph, w.factors, precision=prec)
    try:
        us.debug_set_wait(2_000_000, True)     # about a millisecond, no copy issued
        out = eng.evaluate(w.X)
        st = _status(torch, us, eng)
    finally:
        us.debug_set_wait(0, False)
    assert st == us.USTAT_ERR_DEVICE_TIMEOUT
    assert np.isnan(out["U_sum"]) and np.isnan(out["U_mean"]) and np.all(np.isnan(out["V"]))
    # the same engine and workspace, hook off: correct again
    out = eng.evaluate(w.X)
    assert _status(torch, us, eng) == us.USTAT_OK
    _close(out, uo.ustat(w.graph, w.factors, w.X), 5e-7)


def _nonfinite_cases():
    c4 = synth.workload("c4_rbf", 300)
    p5 = synth.workload("path5_chord_linear_tanh", 257)
    n = 130
    rng = np.random.default_rng(3)
    M = rng.uniform(0.5, 1.5, (n, n))
    vec = rng.uniform(0.5, 1.5, n)
    g_mv = synth.Graph(3, [(0, 1, 0), (1, 2, 0), (2, 0, 0)], [(0, 1)])
    return [
        # the RBF build reading a float64 X directly (its diagonal tiles check it)
        ("rbf-direct", c4.graph, c4.factors, c4.X, "bf16x3", ("X", 137, 5, np.nan)),
        ("rbf-direct-f32", c4.graph, c4.factors, c4.X.astype(np.float32), "fp32", ("X", 299, 31, np.inf)),
        # X converted once (float64 storage)
        ("xconvert", c4.graph, c4.factors, c4.X, "fp64", ("X", 0, 0, -np.inf)),
        ("linear-tanh", p5.graph, p5.factors, p5.X, "bf16x3", ("X", 256, 63, np.nan)),
        # caller matrices and vectors
        ("matrix", g_mv, [synth.Factor(uo.MATRIX, data=M), synth.Factor(uo.VECTOR, data=vec)], np.zeros((n, 1)),
         "bf16x3", ("M", 17, 91, np.inf)),
        ("vector", g_mv, [synth.Factor(uo.MATRIX, data=M), synth.Factor(uo.VECTOR, data=vec)], np.zeros((n, 1)),
         "fp64", ("v", 129, 0, np.nan)),
    ]


@pytest.mark.parametrize("case", range(6))
def test_nonfinite_input_is_reported(env, case):
    torch, engine, us = env
    label, g, facs, X, prec, (where, i, j, bad) = _nonfinite_cases()[case]
    eng = engine.Engine(g, facs, precision=prec)
    clean = eng.evaluate(X)
    assert _status(torch, us, eng) == us.USTAT_OK and np.isfinite(clean["U_sum"]), label
    if where == "X":
        Xb = X.copy()
        Xb[i, j] = bad
        facs_b = facs
    else:
        Xb = X
        facs_b = [synth.Factor(f.kind, f.param, None if f.data is None else np.array(f.data)) for f in facs]
        if where == "M":
            facs_b[0].data[i, j] = bad
        else:
            facs_b[1].data[i] = bad
    eng_b = engine.Engine(g, facs_b, precision=prec)
    out = eng_b.evaluate(Xb)
    assert _status(torch, us, eng_b) == us.USTAT_ERR_NONFINITE, label
    assert np.isnan(out["U_sum"]) and np.all(np.isnan(out["V"])), label
    # a clean evaluation on the same workspace clears the error word
    again = eng_b.evaluate(X) if where == "X" else engine.Engine(g, facs, precision=prec).evaluate(X)
    if where == "X":
        assert _status(torch, us, eng_b) == us.USTAT_OK, label
    assert np.allclose(again["V"], clean["V"], rtol=1e-12, atol=0), label
