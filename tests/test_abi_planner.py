"""Host-side checks of the C ABI: the library builds and loads, exports every
symbol include/ustat.h declares, and its planner (no CUDA call) reproduces the
partition structure the paper fixes.  The oracle's own partition, Moebius and
treewidth functions are the comparison."""
import collections
import json
import os
import re

import pytest

import synth
from oracle import ustat_oracle as uo
from tests.conftest import GOLDEN, ROOT


@pytest.fixture(scope="module")
def us():
    from paper_2508_12627_gb300 import build
    build.build()
    from paper_2508_12627_gb300 import ustat
    return ustat


def test_every_declared_symbol_is_exported(us):
    hdr = open(os.path.join(ROOT, "include", "ustat.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"^\s*(?:const\s+)?(?:int|void|char|size_t)\s*\*?\s*(ustat_\w+)\s*\(", hdr, flags=re.M))
    assert len(names) >= 15
    lib = us.lib()
    for nm in sorted(names):
        assert hasattr(lib, nm), nm
    assert set(us.EXPORTS) == names


def _plan(us, g, kinds, **kw):
    return us.Plan(g, kinds, **kw)


GRAPHS = {
    "triangle": (synth.triangle_graph(), [uo.RBF]),
    "c4": (synth.cycle4_graph(), [uo.RBF]),
    "path5_chord": (synth.path5_chord_graph(), [uo.LINEAR, uo.TANH_DOT]),
    "k4_cycle": (synth.k4_plus_cycle_graph(), [uo.RBF]),
    "c5": (synth.cycle(5), [uo.RBF]),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_partitions_mu_treewidth_match_oracle(us, name):
    g, kinds = GRAPHS[name]
    p = _plan(us, g, kinds, precision="fp64")
    info = p.info
    parts = uo.set_partitions(g.m)
    assert info["n_parts"] == len(parts)
    assert info["rgs"] == parts
    assert info["mu"] == [uo.mu_closed_form(r) for r in parts]
    assert info["tw"] == [uo.treewidth_bruteforce(max(r) + 1, uo.quotient_edges(g, r)) for r in parts]
    ps = _plan(us, g, kinds, precision="fp64", sparsify=True)
    sig = uo.signature(g)
    assert ps.info["evaluated"] == [int(uo.survives(sig, r)) for r in parts]


def test_workload_treewidth_profiles(us):
    # counts of partitions by quotient treewidth for the five workloads (full mode)
    want = {"triangle": {0: 1, 1: 3, 2: 1}, "c4": {0: 1, 1: 9, 2: 5},
            "path5_chord": {0: 1, 1: 31, 2: 20}, "c5": {0: 1, 1: 25, 2: 26},
            "k4_cycle": {0: 1, 1: 48, 2: 128, 3: 26}}
    for name, (g, kinds) in GRAPHS.items():
        p = _plan(us, g, kinds, precision="bf16x3")
        assert dict(collections.Counter(p.info["tw"])) == want[name], name


@pytest.mark.parametrize("m", [4, 5, 6, 7])
def test_chain_N_l_from_planner(us, m):
    # Table 'HOIF_Nl' (Appendix H): N_l of the surviving partitions of a chain
    gold = json.load(open(os.path.join(GOLDEN, "hoif_chain_table.json")))
    p = _plan(us, synth.path(m), [uo.MATRIX], precision="fp64", sparsify=True)
    c = collections.Counter(t for t, e in zip(p.info["tw"], p.info["evaluated"]) if e)
    assert [c.get(l, 0) for l in (1, 2, 3, 4)] == gold["N_l_dp"][str(m)]


def test_sharing_leaves_one_cube_product_for_c4(us):
    # all five treewidth-2 partitions of the 4-cycle reduce against K K^T
    p = _plan(us, synth.cycle4_graph(), [uo.RBF], precision="bf16x3")
    assert p.info["n_gemm"] == 1
    n = 4096
    fp, fn = p.flops(n)
    assert fn == pytest.approx(6 * 2 * n ** 3 + 2 * 2 * n ** 2 * 4 + 4 * n ** 2, rel=0.05)
    assert fp < 1.01 * 2 * n ** 3 + 20 * n ** 2
    q = _plan(us, synth.cycle4_graph(), [uo.RBF], precision="bf16x3", cse=False)
    assert q.info["n_gemm"] >= 5


def test_planners_agree_on_structure(us):
    for name, (g, kinds) in GRAPHS.items():
        a = _plan(us, g, kinds, precision="fp32", planner=us.PLAN_EXHAUSTIVE)
        b = _plan(us, g, kinds, precision="fp32", planner=us.PLAN_MINFILL)
        assert a.info["tw"] == b.info["tw"]
        assert a.flops(1000)[0] <= b.flops(1000)[0] * 1.0001


def test_invalid_graphs_are_rejected(us):
    with pytest.raises(us.UstatError) as e:
        _plan(us, synth.Graph(3, [(0, 3, 0)], []), [uo.RBF])
    assert e.value.code == us.USTAT_ERR_INVALID_ARG
    with pytest.raises(us.UstatError) as e:
        _plan(us, synth.Graph(3, [(0, 1, 0)], []), [uo.RBF])   # vertex 2 not covered
    assert e.value.code == us.USTAT_ERR_INVALID_ARG
    with pytest.raises(us.UstatError) as e:
        _plan(us, synth.path(8), [uo.RBF])
    assert e.value.code == us.USTAT_ERR_UNSUPPORTED
    with pytest.raises(us.UstatError) as e:
        _plan(us, synth.Graph(2, [(0, 1, 0)], []), [uo.TANH_DOT])   # unary kind on an edge
    assert e.value.code == us.USTAT_ERR_INVALID_ARG
    with pytest.raises(us.UstatError) as e:
        _plan(us, synth.complete(5), [uo.RBF])   # K5: treewidth 4
    assert e.value.code == us.USTAT_ERR_TW_TOO_LARGE


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "bf16x4"])
def test_plan_serialisation_round_trip(us, name, prec):
    g, kinds = GRAPHS[name]
    p = _plan(us, g, kinds, precision=prec)
    p.set_variant(17, 1)
    data = p.to_bytes()
    q = us.Plan.from_bytes(data, g, kinds, prec)
    assert q.describe() == p.describe() and q.info == p.info
    assert q.flops(3000) == p.flops(3000) and q.workspace_bytes(3000, 16) == p.workspace_bytes(3000, 16)
    assert us.plan_orders(q) == us.plan_orders(p)
    assert q.to_bytes() == data


def test_plan_deserialisation_refuses_other_bytes(us):
    g, kinds = GRAPHS["k4_cycle"]
    data = _plan(us, g, kinds).to_bytes()
    bad = [b"", data[:-1], data + b"\0", b"XXXX" + data[4:], data[:8] + bytes([data[8] ^ 1]) + data[9:]]
    # the first operation's output slot pointed past the plan's slots: after the
    # 64-byte header come the factor kinds and the 8-byte slots, each a count and
    # its records, then the operations (kind, factor, out, ...)
    import struct
    nf = struct.unpack_from("<Q", data, 64)[0]
    ns = struct.unpack_from("<Q", data, 72 + 4 * nf)[0]
    at = 72 + 4 * nf + 8 + 8 * ns + 8 + 8
    assert struct.unpack_from("<i", data, at)[0] in range(ns)
    bad.append(data[:at] + struct.pack("<i", ns + 5) + data[at + 4:])
    for blob in bad:
        with pytest.raises(us.UstatError) as e:
            us.Plan.from_bytes(blob, g, kinds, "bf16x3")
        assert e.value.code == us.USTAT_ERR_INVALID_ARG


def test_status_rejects_a_missing_workspace(us):
    # argument checks come before any CUDA call
    with pytest.raises(us.UstatError) as e:
        us.status(0, 0)
    assert e.value.code == us.USTAT_ERR_INVALID_ARG


def test_factor_matrix_argument_checks(us):
    # rejected on the host before any CUDA call: a kind the call does not build,
    # a non-integer or out-of-range column count, a NULL or unaligned workspace
    for kind, param, ws in [(us.RBF, 1.0, 256), (us.MATRIX, 1.0, 256), (us.DIST, 2.5, 256),
                            (us.LOWRANK, 0.0, 256), (us.DIST, 5000.0, 256), (us.DIST, 3.0, 0),
                            (us.COMPLEMENT, 1.0, 128)]:
        with pytest.raises(us.UstatError) as e:
            us.factor_matrix(kind, param, 4096, 10, 8192, ws, 0)
        assert e.value.code == us.USTAT_ERR_INVALID_ARG, (kind, param, ws)


def test_workspace_bytes_scale(us):
    p = _plan(us, synth.cycle4_graph(), [uo.RBF], precision="bf16x3")
    a, b = p.workspace_bytes(1000, 32), p.workspace_bytes(2000, 32)
    assert 3.5 < b / a < 4.5
    assert p.host_staging_bytes(1000, 32) >= 8 * 1000 * 32


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16x3", "bf16x4", "bf16x5"])
def test_every_plan_is_well_formed(us, prec):
    # ustat_plan checks that every slot an operation reads is written by an earlier
    # operation and that every partition's scalars are produced; it returns an
    # error otherwise.  Sweep graphs, modes and options.
    graphs = [(synth.cycle4_graph(), [uo.RBF]), (synth.triangle_graph(), [uo.RBF]),
              (synth.path5_chord_graph(), [uo.LINEAR, uo.TANH_DOT]), (synth.k4_plus_cycle_graph(), [uo.RBF]),
              (synth.cycle(5), [uo.RBF]), (synth.path(7), [uo.MATRIX]),
              (synth.Graph(4, [(0, 1, 0), (2, 1, 2), (2, 3, 0), (3, 0, 2), (0, 2, 0)], [(1, 1)]),
               [uo.MATRIX, uo.VECTOR, uo.MATRIX])]
    for g, kinds in graphs:
        for sp in (False, True):
            for cse in (False, True):
                for pl in (us.PLAN_EXHAUSTIVE, us.PLAN_MINFILL):
                    p = us.Plan(g, kinds, precision=prec, sparsify=sp, cse=cse, planner=pl)
                    assert p.info["n_parts"] == len(uo.set_partitions(g.m))


def test_engine_plan_cache(us, tmp_path):
    # planning only (no device work): the second engine reads the plan the first wrote
    from paper_2508_12627_gb300 import engine
    w = synth.workload("k4_cycle_rbf", 16)
    a = engine.Engine(w.graph, w.factors, precision="bf16x3", plan_cache=str(tmp_path))
    b = engine.Engine(w.graph, w.factors, precision="bf16x3", plan_cache=str(tmp_path))
    c = engine.Engine(w.graph, w.factors, precision="bf16x4", plan_cache=str(tmp_path))
    assert not a.plan_cached and b.plan_cached and not c.plan_cached
    assert b.plan.describe() == a.plan.describe() and b.n_parts == a.n_parts == 203
    assert len(list(tmp_path.iterdir())) == 2

