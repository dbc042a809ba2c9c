"""ustat_eval_noalloc (the evaluation that allocates nothing and runs in the
library's own fixed device scratch) against ustat_eval with a caller workspace,
on the same plan and inputs: a set-up call and two calls in a row, each within the parity
tolerance of the workspace path, plus the size limit.  The file name sorts last
so that it also runs after every other GPU test has used the device."""
import numpy as np
import pytest

import synth
from oracle import ustat_oracle as uo

# relative to the sum of absolute terms; both paths run the same kernels, only the
# order of floating-point atomic additions may differ between two runs
SAME_PATH_TOL = 1e-12


@pytest.fixture(scope="module")
def us():
    from paper_2508_12627_gb300 import build
    build.build()
    from paper_2508_12627_gb300 import ustat
    return ustat


def test_oversize_request_is_rejected_before_any_device_work(us):
    w = synth.workload("c4_rbf", 8)
    p = us.Plan(w.graph, [f.kind for f in w.factors], precision="bf16x3")
    n = 8192
    assert p.workspace_bytes(n, 32) > us.NOALLOC_MAX_BYTES
    with pytest.raises(us.UstatError) as e:
        # X and the outputs are never touched: the size check comes first
        us.ustat_eval_noalloc(p, 256, 0, n, 32, [(f.kind, f.param, 0) for f in w.factors], None, 256, 256)
    assert e.value.code == us.USTAT_ERR_WORKSPACE


@pytest.mark.gpu
@pytest.mark.parametrize("name,n,prec", [("c4_rbf", 1000, "bf16x3"), ("k4_cycle_rbf", 100, "bf16x3"),
                                         ("path5_chord_linear_tanh", 600, "fp32"), ("triangle_rbf", 200, "fp64")])
def test_noalloc_matches_workspace_path(us, name, n, prec):
    import torch
    from paper_2508_12627_gb300 import engine
    w = synth.workload(name, n)
    eng = engine.Engine(w.graph, w.factors, precision=prec)
    X = eng.to_device(w.X)
    assert eng.plan.workspace_bytes(n, X.shape[1]) <= us.NOALLOC_MAX_BYTES
    k = eng.n_parts
    ref = torch.empty(2 + k, dtype=torch.float64, device=X.device)
    eng.launch(X, ref)
    facs = eng.factor_tuples(n)
    st = torch.cuda.current_stream(X.device).cuda_stream
    outs = [torch.full((2 + k,), float("nan"), dtype=torch.float64, device=X.device) for _ in range(3)]

    def call(o):
        us.ustat_eval_noalloc(eng.plan, X.data_ptr(), 0 if X.dtype == torch.float64 else 1, n, X.shape[1], facs,
                              st, o.data_ptr(), o.data_ptr() + 16)

    # the first call on a device is the set-up: the driver may load the library's
    # device image, scratch array included, at that point
    call(outs[0])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(X.device)[0]
    call(outs[1])
    call(outs[2])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(X.device)[0] >= free0   # the two calls in a row took no device memory
    a = uo.ustat(w.graph, w.factors, w.X, absolute=True)
    Vabs = np.maximum(np.array(a["V"]), 1e-300)
    mu = np.array(a["mu"], dtype=np.float64)
    uabs = float(np.abs(mu) @ np.array(a["V"]))
    r = ref.cpu().numpy()
    for o in outs:
        o = o.cpu().numpy()
        assert np.all(np.abs(o[2:] - r[2:]) <= SAME_PATH_TOL * Vabs), (name, np.abs(o[2:] - r[2:]) / Vabs)
        assert abs(o[0] - r[0]) <= SAME_PATH_TOL * uabs
        assert o[1] == pytest.approx(r[1], rel=1e-10, abs=SAME_PATH_TOL * uabs)


@pytest.mark.gpu
def test_noalloc_status_codes_on_device(us):
    # n < m is reported, as by ustat_eval
    import torch
    w = synth.workload("c4_rbf", 3)
    p = us.Plan(w.graph, [f.kind for f in w.factors], precision="bf16x3")
    X = torch.as_tensor(np.ascontiguousarray(w.X), device="cuda:0")
    out = torch.empty(2 + p.info["n_parts"], dtype=torch.float64, device="cuda:0")
    with pytest.raises(us.UstatError) as e:
        us.ustat_eval_noalloc(p, X.data_ptr(), 0, 3, X.shape[1], [(f.kind, f.param, 0) for f in w.factors],
                              torch.cuda.current_stream().cuda_stream, out.data_ptr(), out.data_ptr() + 16)
    assert e.value.code == us.USTAT_ERR_N_LT_M
