"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element
by element (U_sum, U_mean and every V_pi), on seeded inputs that span several
128 x 128 tiles and a ragged tail, plus edge cases.

Tolerances (relative to the oracle's sum of absolute terms V_abs, which equals
|V| for positive kernels such as the RBF):
  fp64    1e-11   (float64 throughout; only summation order differs)
  bf16x3  1e-8 at the workloads' own sizes (the engine's accuracy target) on
          kernels with bounded rows (RBF); 1e-6 on the heavy-tailed linear
          workload, whose rows span a wide range (fixed-point slices relative to
          the row maximum lose bits on small entries)
  bf16x4  1e-8 at every size (four slices; matrices stored and reduced in
          float64, the mode for data of wide dynamic range)
  fp32    1e-8 at the workloads' own sizes
  tf32    2e-2    (10-bit mantissa operands: reported, not a target)
At small n (edge cases, ragged tiles) the float32-storage paths are held to
SMALL_N = 5e-7: every factor entry is stored in float32 (relative rounding
<= 2^-24) and a term multiplies at most |E| <= 7 entries, so every term, and
hence V_pi (a weighted mean of terms), is within 7 * 2^-24 = 4.2e-7; the 1e-8
target relies on these independent roundings averaging out over many terms.
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import ustat_oracle as uo

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "bf16x3": 1e-8, "bf16x4": 1e-8, "bf16x5": 1e-8, "fp32": 1e-8, "tf32": 2e-2}
SMALL_N = 5e-7
WIDE_RANGE = {"path5_chord_linear_tanh"}
FULL_SIZE = {"triangle_rbf": 200, "c4_rbf": 4096, "path5_chord_linear_tanh": 16384, "k4_cycle_rbf": 1024}


def tol_for(name, prec, n=None):
    if prec == "bf16x3" and name in WIDE_RANGE:
        return 1e-6
    if prec in ("bf16x3", "fp32") and n is not None and n < FULL_SIZE.get(name, 0):
        return SMALL_N
    # bf16x4 stores every matrix in float64 and reduces in float64: 1e-8 at any n
    return TOL[prec]


@pytest.fixture(scope="module")
def eng_mod():
    import torch
    assert torch.cuda.is_available()
    from paper_2508_12627_gb300 import build
    build.build()
    from paper_2508_12627_gb300 import engine
    return engine


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _stored(name):
    """The oracle's values for a workload at its full size, written by
    tests/golden/make_workload_golden.py (FP64 partition sum on synth's inputs)."""
    with open(os.path.join(GOLDEN, "workload_%s.json" % name)) as f:
        g = json.load(f)
    return {"V": g["V"], "mu": g["mu"], "U_sum": g["U_sum"], "U_mean": g["U_mean"]}, {"V": g["V_abs"]}


def _oracle(w, sparse=False):
    r = uo.ustat(w.graph, w.factors, w.X, sparse=sparse)
    a = uo.ustat(w.graph, w.factors, w.X, sparse=sparse, absolute=True)
    return r, a


def _compare(out, ref, absref, tol, label):
    Vabs = np.array(absref["V"])
    V = np.array(ref["V"])
    err = np.abs(out["V"] - V)
    bad = err > tol * np.maximum(Vabs, 1e-300)
    assert not bad.any(), (label, np.argwhere(bad).ravel()[:5], (err / np.maximum(Vabs, 1e-300)).max())
    uabs = sum(abs(mu) * va for mu, va in zip(ref["mu"], absref["V"]))
    assert abs(out["U_sum"] - ref["U_sum"]) <= tol * uabs, (label, out["U_sum"], ref["U_sum"])
    if ref["U_sum"] != 0.0:
        # U_mean = U_sum / (n)_m: the same relative agreement
        ratio_out = out["U_mean"] / out["U_sum"]
        ratio_ref = ref["U_mean"] / ref["U_sum"]
        assert ratio_out == pytest.approx(ratio_ref, rel=1e-14), label


CASES = [("triangle_rbf", 200), ("c4_rbf", 300), ("path5_chord_linear_tanh", 257), ("k4_cycle_rbf", 72)]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "bf16x4", "bf16x5", "fp32", "tf32"])
@pytest.mark.parametrize("name,n", CASES)
def test_workloads_against_oracle(eng_mod, name, n, prec):
    w = synth.workload(name, n=n)
    ref, absref = _oracle(w)
    eng = eng_mod.Engine(w.graph, w.factors, precision=prec)
    out = eng.evaluate(w.X)
    _compare(out, ref, absref, tol_for(name, prec, n), "%s n=%d %s" % (name, n, prec))


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x4", "bf16x5", "tf32", "fp32"])
def test_heavy_tailed_matrix_factor(eng_mod, prec):
    # a symmetric Student-t(2) matrix factor: rows with a very wide dynamic range
    n = 512
    A = np.random.default_rng(5).standard_t(2, (n, n))
    A = (A + A.T) / 2
    facs = [synth.Factor(uo.MATRIX, data=A)]
    g = synth.triangle_graph()
    X = np.zeros((n, 1))
    ref, absref = uo.ustat(g, facs, X), uo.ustat(g, facs, X, absolute=True)
    out = eng_mod.Engine(g, facs, precision=prec).evaluate(X)
    tol = {"bf16x3": 1e-6, "bf16x4": SMALL_N, "bf16x5": SMALL_N, "tf32": 2e-2, "fp32": SMALL_N}[prec]
    _compare(out, ref, absref, tol, "t2 %s" % prec)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "bf16x4"])
@pytest.mark.parametrize("n", [4, 5, 64, 127, 128, 129, 256, 385, 1100, 2049, 2500])
def test_c4_sizes_and_ragged_tails(eng_mod, n, prec):
    # n = 2049 and 2500: the RBF build's last partial wave runs as column halves
    # (2500: 58 tiles in halves, the last column block 68 columns wide)
    w = synth.workload("c4_rbf", n=n)
    ref, absref = _oracle(w)
    eng = eng_mod.Engine(w.graph, w.factors, precision=prec)
    eng.workspace(eng.plan.workspace_bytes(n, w.X.shape[1])).fill_(255)   # NaN bytes: no stale reads
    out = eng.evaluate(w.X)
    _compare(out, ref, absref, tol_for("c4_rbf", prec, n), "c4 n=%d %s" % (n, prec))


def rank1_values(graph, u):
    """V_pi for K = u u^T on every edge and the unary factor u, in closed form:
    prod over the blocks B of pi of p_deg(B)(u), p_k = sum_i u_i^k, deg(B) the
    number of factor slots (edge endpoints, unary factors) landing in B; and
    U_sum = sum_pi mu_pi V_pi (exact integers)."""
    ps = {}
    V, U = [], 0
    for rgs in uo.set_partitions(graph.m):
        deg = [0] * (max(rgs) + 1)
        for a, b, _ in graph.edges:
            deg[rgs[a]] += 1
            deg[rgs[b]] += 1
        for a, _ in graph.unary:
            deg[rgs[a]] += 1
        v = 1
        for k in deg:
            if k not in ps:
                ps[k] = int(np.sum(u.astype(np.int64) ** k))
            v *= ps[k]
        V.append(v)
        U += uo.mu_closed_form(rgs) * v
    return V, U


def sparse_ternary(n, nnz, seed):
    """u with exactly nnz entries of +-1 at random positions, 0 elsewhere: the power
    sums stay small, so every partial sum of the float32 paths is an exact integer."""
    rng = np.random.default_rng(seed)
    u = np.zeros(n)
    u[rng.choice(n, nnz, replace=False)] = rng.choice([-1.0, 1.0], nnz)
    return u


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "bf16x4"])
@pytest.mark.parametrize("n", [5, 64, 127, 129, 200, 385, 1100, 2049])
def test_rank1_integer_factors_bit_exact(eng_mod, prec, n):
    # K = u u^T with u in {-1, 0, 1}: every partial sum is an integer below 2^24,
    # so the float32 and split bf16 paths are exact too -- at every ragged size
    u = synth.ternary_vector(n, 9) if n <= 64 else sparse_ternary(n, 40, 9)
    facs = [synth.Factor(uo.MATRIX, data=np.outer(u, u)), synth.Factor(uo.VECTOR, data=u)]
    graphs = [synth.cycle4_graph(), synth.path5_chord_graph(), synth.triangle_graph()]
    if prec in ("bf16x3", "bf16x4") and 6 <= n <= 385:
        graphs.append(synth.k4_plus_cycle_graph())
    for g in graphs:
        V, U = rank1_values(g, u)
        eng = eng_mod.Engine(g, facs, precision=prec)
        eng.workspace(eng.plan.workspace_bytes(n, 1)).fill_(255)   # NaN bytes: no stale reads
        out = eng.evaluate(np.zeros((n, 1)))
        assert list(out["V"]) == [float(v) for v in V], (prec, n, g.m)
        assert out["U_sum"] == float(U)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("n", [150, 200, 452])
def test_asymmetric_matrix_factors(eng_mod, prec, n):
    # caller-supplied asymmetric factors with mixed orientations (transposed reads);
    # n = 200 and 452 (multiples of 4, ragged 64-row tiles) take the streaming
    # reduction in float32 and float64, n = 150 the float32 tile kernel
    rng = np.random.default_rng(21)
    facs = [synth.Factor(uo.MATRIX, data=rng.uniform(0.2, 1.0, (n, n))),
            synth.Factor(uo.VECTOR, data=rng.uniform(0.5, 1.5, n)),
            synth.Factor(uo.MATRIX, data=rng.uniform(0.2, 1.0, (n, n)))]
    g = synth.Graph(4, [(0, 1, 0), (2, 1, 2), (2, 3, 0), (3, 0, 2), (0, 2, 0)], [(1, 1)])
    X = np.zeros((n, 1))
    ref = uo.ustat(g, facs, X)
    out = eng_mod.Engine(g, facs, precision=prec).evaluate(X)
    _compare(out, ref, ref, tol_for("asym", prec, 0) if prec == "fp64" else SMALL_N, "asym %s" % prec)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "bf16x4", "bf16x5"])
def test_sparse_mode_and_sharing_and_planners_agree(eng_mod, prec):
    w = synth.workload("path5_chord_linear_tanh", n=200)
    ref, absref = _oracle(w)
    uabs = sum(abs(mu) * va for mu, va in zip(ref["mu"], absref["V"]))
    from paper_2508_12627_gb300 import ustat as us
    outs = [eng_mod.Engine(w.graph, w.factors, precision=prec, sparsify=sp, cse=cse, planner=pl).evaluate(w.X)
            for sp in (False, True) for cse in (False, True) for pl in (us.PLAN_EXHAUSTIVE, us.PLAN_MINFILL)]
    for o in outs:
        assert abs(o["U_sum"] - ref["U_sum"]) <= tol_for(w.name, prec, w.n) * uabs


@pytest.mark.parametrize("name", ["rbf", "linear", "rbf-near-pairs"])
def test_kernel_matrix_sum_has_no_bias(eng_mod, name):
    # m = 2, one edge: U_sum = sum_{i != j} F(x_i, x_j).  A mean bias of the device's
    # float32 kernel entries would show at full size (16.7M terms); symmetric
    # rounding errors average out far below the split path's 1e-8 target.  With
    # near pairs (every odd row a 1e-4 perturbation of the row before) the Gram
    # form's squared distances cancel to ~1e-7 of the norms on half the rows.
    n, d = 4096, 32
    X = synth.normal_X(n, d, 3)
    if name == "rbf-near-pairs":
        X[1::2] = X[0::2] + 1e-4 * synth.normal_X(n // 2, d, 4)
    g = synth.Graph(2, [(0, 1, 0)], [])
    f = [synth.linear(d)] if name == "linear" else [synth.rbf(d)]
    ref, absref = _oracle(synth.Workload("m2", g, f, n, d, X))
    for prec in ("fp32", "bf16x3"):
        out = eng_mod.Engine(g, f, precision=prec).evaluate(X)
        uabs = sum(abs(mu) * va for mu, va in zip(ref["mu"], absref["V"]))
        assert abs(out["U_sum"] - ref["U_sum"]) <= 1e-9 * uabs, (name, prec, out["U_sum"], ref["U_sum"])


def test_status_after_an_evaluation_is_ok(eng_mod):
    import torch
    from paper_2508_12627_gb300 import ustat as us
    w = synth.workload("c4_rbf", 300)
    eng = eng_mod.Engine(w.graph, w.factors, precision="bf16x3")
    out = eng.evaluate(w.X)
    assert np.isfinite(out["U_sum"])
    assert us.status(eng._ws.data_ptr(), torch.cuda.current_stream().cuda_stream) == us.USTAT_OK


def test_n_smaller_than_m_is_an_error(eng_mod):
    from paper_2508_12627_gb300 import ustat as us
    w = synth.workload("c4_rbf", n=3)
    with pytest.raises(us.UstatError) as e:
        eng_mod.Engine(w.graph, w.factors, precision="bf16x3").evaluate(w.X)
    assert e.value.code == us.USTAT_ERR_N_LT_M


def test_row_permutation_invariance_on_gpu(eng_mod):
    w = synth.workload("c4_rbf", n=333)
    e = eng_mod.Engine(w.graph, w.factors, precision="bf16x3")
    a = e.evaluate(w.X)
    b = e.evaluate(w.X[np.random.default_rng(1).permutation(333)])
    assert np.allclose(a["V"], b["V"], rtol=SMALL_N, atol=0)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x4"])
def test_c4_full_size_against_oracle(eng_mod, prec):
    # the 4-cycle RBF workload at n = 4096, d = 32, in the launch configuration the
    # benchmark times: all 15 V_pi and U against the FP64 oracle's stored values
    w = synth.workload("c4_rbf")
    ref, absref = _stored("c4_rbf")
    eng = eng_mod.Engine(w.graph, w.factors, precision=prec)
    eng.workspace(eng.plan.workspace_bytes(w.n, w.d)).fill_(255)   # NaN bytes: no stale reads
    out = eng.evaluate(w.X)
    _compare(out, ref, absref, 1e-8, "c4 full " + prec)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "bf16x4", "fp32"])
def test_triangle_full_size_against_oracle(eng_mod, prec):
    # the triangle workload at its size n = 200 (every partition) in every 1e-8 mode
    w = synth.workload("triangle_rbf")
    ref, absref = _stored("triangle_rbf")
    out = eng_mod.Engine(w.graph, w.factors, precision=prec).evaluate(w.X)
    _compare(out, ref, absref, TOL[prec], "triangle full " + prec)


K4C_N = 200


@pytest.fixture(scope="module")
def k4c_ref():
    # K4 + cycle at n = 200 (two 128-row tiles with a ragged tail): all 203
    # partitions, 26 of them treewidth 3, which the oracle evaluates in seconds
    w = synth.workload("k4_cycle_rbf", K4C_N)
    return w, uo.ustat(w.graph, w.factors, w.X)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x4", "bf16x5", "fp32"])
def test_k4_cycle_treewidth3_steps_multi_tile(eng_mod, k4c_ref, prec):
    # the s = 3 steps (tensor cores in the split modes) against the oracle element
    # by element (RBF factors are positive: V_abs = V)
    w, ref = k4c_ref
    eng = eng_mod.Engine(w.graph, w.factors, precision=prec)
    eng.workspace(eng.plan.workspace_bytes(w.n, w.d)).fill_(255)   # NaN bytes: no stale reads
    out = eng.evaluate(w.X)
    _compare(out, ref, ref, tol_for("k4_cycle_rbf", prec, K4C_N), "k4+cycle n=200 " + prec)


# K4 + cycle at its full size n = 1024: 203 partitions, 26 of treewidth 3, whose
# s = 3 steps run in 25 batches of 42 indices, each split on the caller's stream
# into one of two alternating regions while the GEMM of the batch before runs on
# a second stream.  Every split mode meets 1e-8 here: the products of entrywise
# powers of K (dominant diagonals) are split without their diagonals, whose
# terms the GEMM epilogue adds exactly.
@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-8), ("bf16x4", 1e-8), ("bf16x5", 1e-8)])
def test_k4_cycle_full_size_against_oracle(eng_mod, prec, tol):
    w = synth.workload("k4_cycle_rbf")
    ref, absref = _stored("k4_cycle_rbf")
    eng = eng_mod.Engine(w.graph, w.factors, precision=prec)
    eng.workspace(eng.plan.workspace_bytes(w.n, w.d)).fill_(255)   # NaN bytes: no stale reads
    out = eng.evaluate(w.X)
    tw = eng.plan.info["tw"]
    assert sum(1 for t in tw if t == 3) == 26
    _compare(out, ref, absref, tol, "k4+cycle full " + prec)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x4"])
def test_k4_cycle_full_size_rank1_bit_exact(eng_mod, prec):
    # the same graph and size with K = u u^T (48 nonzero +-1 entries): the 25
    # batches, both split regions and both streams give the exact integers
    n = 1024
    g = synth.k4_plus_cycle_graph()
    u = sparse_ternary(n, 48, 11)
    facs = [synth.Factor(uo.MATRIX, data=np.outer(u, u))]
    V, U = rank1_values(g, u)
    eng = eng_mod.Engine(g, facs, precision=prec)
    eng.workspace(eng.plan.workspace_bytes(n, 1)).fill_(255)
    out = eng.evaluate(np.zeros((n, 1)))
    assert list(out["V"]) == [float(v) for v in V]
    assert out["U_sum"] == float(U)


def test_path5_full_size_rank1_bit_exact(eng_mod):
    # the path + chord graph at its full size n = 16384 with K = u u^T and the
    # unary factor u (200 nonzero +-1 entries), bf16x3: its treewidth-2 products
    # on the tensor cores give the exact integers
    n = 16384
    g = synth.path5_chord_graph()
    u = sparse_ternary(n, 200, 12)
    facs = [synth.Factor(uo.MATRIX, data=np.outer(u, u)), synth.Factor(uo.VECTOR, data=u)]
    V, U = rank1_values(g, u)
    out = eng_mod.Engine(g, facs, precision="bf16x3").evaluate(np.zeros((n, 1)))
    assert list(out["V"]) == [float(v) for v in V]
    assert out["U_sum"] == float(U)


@pytest.mark.parametrize("prec,tol", [("bf16x4", 1e-8), ("bf16x5", 1e-8), ("bf16x3", 2e-7)])
def test_path5_full_size_against_oracle(eng_mod, prec, tol):
    # the path + chord workload at its full size, n = 16384, d = 64, t(5) data: all
    # 52 V_pi (20 of them treewidth-2 products on the tensor cores) and U against
    # the oracle's stored values.  The float64-storage modes meet 1e-8; bf16x3
    # stores the products of these heavy-tailed rows in float32, the float32
    # CUDA-core mode's class (1.1e-7 measured for that mode)
    w = synth.workload("path5_chord_linear_tanh")
    ref, absref = _stored("path5_chord_linear_tanh")
    out = eng_mod.Engine(w.graph, w.factors, precision=prec).evaluate(w.X)
    _compare(out, ref, absref, tol, "path5 full " + prec)


@pytest.mark.parametrize("prec,shape", [("bf16x3", 0), ("bf16x3", 1), ("bf16x3", 2), ("bf16x4", 0), ("bf16x4", 2),
                                        ("bf16x5", 2)])
@pytest.mark.parametrize("name,n", [("c4_rbf", 300), ("path5_chord_linear_tanh", 257), ("k4_cycle_rbf", 72)])
def test_gemm_tile_variants(eng_mod, name, n, prec, shape):
    # every tensor-core tile shape and raster group the autotuner may pick gives the
    # oracle's result within the mode's tolerance
    w = synth.workload(name, n)
    ref, absref = _oracle(w)
    for gr in (0, 3):
        eng = eng_mod.Engine(w.graph, w.factors, precision=prec)
        eng.plan.set_variant(gr | (shape << 2))
        out = eng.evaluate(w.X)
        _compare(out, ref, absref, tol_for(name, prec, n), (name, prec, shape, gr))


def test_wide_narrow_tiles_double_buffered(eng_mod):
    # bf16x4 with 128 x 64 tiles keeps two accumulator sets in TMEM: at n = 2500 a
    # CTA runs several tiles, so both sets and their barriers are used
    w = synth.workload("c4_rbf", 2500)
    ref, absref = _oracle(w)
    eng = eng_mod.Engine(w.graph, w.factors, precision="bf16x4")
    eng.plan.set_variant(0)
    out = eng.evaluate(w.X)
    _compare(out, ref, absref, 1e-8, "c4 n=2500 bf16x4 shape 0")


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
@pytest.mark.parametrize("name,n", [("c4_rbf", 5), ("c4_rbf", 63), ("c4_rbf", 65), ("c4_rbf", 129), ("c4_rbf", 300),
                                    ("triangle_rbf", 200), ("k4_cycle_rbf", 72)])
def test_rbf_build_tile_variants(eng_mod, name, n, prec):
    # every form of the RBF kernel-matrix build: the tensor-core Gram build (the
    # default, variant 0) and the CUDA-core direct-difference build on 128 x 128 or
    # 64 x 64 tiles (bits 5 and 4 of the plan variant): tiles, mirror, digit
    # planes and fused reductions against the oracle
    w = synth.workload(name, n)
    ref, absref = _oracle(w)
    for variant in (0, 32, 48):
        eng = eng_mod.Engine(w.graph, w.factors, precision=prec)
        eng.plan.set_variant(variant)
        # every workspace byte 0xff (a NaN in float32 and float64): a read of
        # anything the evaluation did not write shows up in the result
        eng.workspace(eng.plan.workspace_bytes(n, w.X.shape[1])).fill_(255)
        out = eng.evaluate(w.X)
        _compare(out, ref, absref, tol_for(name, prec, n), (name, n, prec, variant))


@pytest.mark.parametrize("prec", ["bf16x3", "fp32", "bf16x4"])
def test_input_dtype_and_alignment(eng_mod, prec):
    # X given as float64 or float32, at a 16-byte aligned address or 8 bytes off it
    # (the RBF build reads the caller's X directly in the float32-storage modes)
    import torch
    from paper_2508_12627_gb300 import ustat as us
    n = 300
    w = synth.workload("c4_rbf", n)
    ref, absref = _oracle(w)
    eng = eng_mod.Engine(w.graph, w.factors, precision=prec)
    d = w.X.shape[1]
    for dt in (torch.float64, torch.float32):
        x32 = torch.as_tensor(w.X).to(dt)
        if dt == torch.float32:
            # the oracle on the float32-rounded data
            w2 = synth.Workload(w.name, w.graph, w.factors, n, d, x32.double().numpy())
            r, ra = _oracle(w2)
        else:
            r, ra = ref, absref
        for off in (0, 1):
            buf = torch.empty(n * d + 2, dtype=dt, device="cuda")
            X = buf[off:off + n * d].view(n, d)
            X.copy_(x32)
            out = torch.empty(2 + eng.n_parts, dtype=torch.float64, device="cuda")
            ws = eng.workspace(eng.plan.workspace_bytes(n, d))
            us.ustat_eval(eng.plan, X.data_ptr(), 0 if dt == torch.float64 else 1, n, d, eng.factor_tuples(n),
                          ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream, out.data_ptr(),
                          out.data_ptr() + 16)
            o = out.cpu().numpy()
            _compare({"U_sum": o[0], "U_mean": o[1], "V": o[2:]}, r, ra, tol_for("c4_rbf", prec, n),
                     (prec, str(dt), off))


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "bf16x4"])
@pytest.mark.parametrize("n", [5, 130, 300])
def test_device_built_factor_kinds(eng_mod, n, prec):
    # the factors the library builds from caller data (DIST, LOWRANK, COMPLEMENT,
    # GRAM) on a 4-vertex kernel graph that uses all four, with a ragged tail,
    # against the oracle's definitions of the same factors
    rng = np.random.default_rng(40 + n)
    Y = rng.standard_normal((n, 5))
    PQ = rng.uniform(0.2, 1.0, (n, 6))
    A = (rng.random((n, n)) < 0.3).astype(float)
    facs = [synth.Factor(synth.DIST, 5.0, Y), synth.Factor(synth.LOWRANK, 3.0, PQ),
            synth.Factor(synth.COMPLEMENT, 1.0, A), synth.Factor(synth.GRAM, 4.0, PQ[:, 1:5].copy())]
    g = synth.Graph(4, [(0, 1, 0), (1, 2, 1), (2, 3, 2), (3, 0, 1), (0, 2, 0), (1, 3, 3)], [])
    X = np.zeros((n, 1))
    ref, absref = uo.ustat(g, facs, X), uo.ustat(g, facs, X, absolute=True)
    out = eng_mod.Engine(g, facs, precision=prec).evaluate(X)
    _compare(out, ref, absref, 1e-11 if prec == "fp64" else (1e-8 if prec == "bf16x4" else SMALL_N),
             "kinds n=%d %s" % (n, prec))


@pytest.mark.parametrize("n", [5, 130, 300])
def test_factor_matrix_entry_point(eng_mod, n):
    # ustat_factor_matrix against the oracle's definitions of the three factors
    import torch
    from paper_2508_12627_gb300 import ustat as us
    rng = np.random.default_rng(70 + n)
    Y = rng.standard_normal((n, 5))
    PQ = rng.uniform(-1.0, 1.0, (n, 6))
    A = (rng.random((n, n)) < 0.3).astype(float)
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    for kind, param, data in [(us.DIST, 5.0, Y), (us.LOWRANK, 3.0, PQ), (us.COMPLEMENT, 1.0, A),
                              (us.GRAM, 4.0, PQ[:, 1:5].copy())]:
        dd = torch.from_numpy(np.ascontiguousarray(data)).cuda()
        F = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        us.factor_matrix(kind, param, dd.data_ptr(), n, F.data_ptr(), ws.data_ptr(), st)
        assert us.status(ws.data_ptr(), st) == us.USTAT_OK
        want = uo.factor_tensor(kind, np.zeros((n, 1)), param, data)
        got = F.cpu().numpy()
        if kind == us.COMPLEMENT:
            assert np.array_equal(got, want)
        else:
            # a sum of r float64 terms in another order: a few ulps of the scale
            if kind == us.DIST:
                scale = (np.abs(Y) ** 2).sum(1).max() ** 0.5 * 2
            elif kind == us.LOWRANK:
                scale = np.abs(PQ[:, :3]).max(1)[:, None] * np.abs(PQ[:, 3:]).max(1)[None, :] * 3
            else:
                scale = 4 * np.abs(data).max() ** 2
                assert np.array_equal(got, got.T)   # declared symmetric: exactly
            assert np.all(np.abs(got - want) <= 1e-14 * scale), kind
    # a NaN in the data: the status word says so
    Y[n // 2, 1] = np.nan
    dd = torch.from_numpy(Y).cuda()
    F = torch.empty((n, n), dtype=torch.float64, device="cuda")
    us.factor_matrix(us.DIST, 5.0, dd.data_ptr(), n, F.data_ptr(), ws.data_ptr(), st)
    assert us.status(ws.data_ptr(), st) == us.USTAT_ERR_NONFINITE
