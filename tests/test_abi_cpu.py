"""CPU-only checks of the C ABI: the library loads, exports every symbol the
header declares, validates arguments, and the host planner (tn_plan makes no
CUDA call) produces consistent plans."""
import math
import os
import re

import numpy as np
import pytest

import rqcgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tn():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_01066_gb300 import tn as _tn
    return _tn


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "tn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(tn):
    lib = tn.load()
    syms = _declared_symbols()
    assert len(syms) >= 14
    for s in syms:
        assert hasattr(lib, s), f"missing export {s}"
        assert s in tn._SIGS, f"binding lacks {s}"


def test_network_argument_errors(tn):
    lib = tn.load()
    import ctypes
    h = ctypes.c_void_p()
    assert lib.tn_network_from_circuit(None, ctypes.byref(h)) == tn.TN_ERR_ARG
    assert b"NULL" in lib.tn_last_error()
    bad = tn.tn_circuit(0, 0, None, None, None)
    assert lib.tn_network_from_circuit(ctypes.byref(bad), ctypes.byref(h)) == tn.TN_ERR_ARG
    q = (ctypes.c_int32 * 2)(0, 0)       # a gate acting twice on qubit 0
    m = (ctypes.c_double * 32)()
    c = tn.tn_circuit(2, 1, q, m, None)
    assert lib.tn_network_from_circuit(ctypes.byref(c), ctypes.byref(h)) == tn.TN_ERR_ARG


def test_plan_options_validated(tn):
    circ, om, _ = rqcgen.config_circuit("c1")
    net = tn.Network(circ)
    with pytest.raises(tn.TnError) as e:
        tn.Plan(net, open_mask=om, precision=7)
    assert e.value.status == tn.TN_ERR_ARG
    with pytest.raises(tn.TnError):
        tn.Plan(net, open_mask=om, complex_mult=5)
    with pytest.raises(tn.TnError) as e:
        tn.Plan(net, open_mask=om, complex_mult=3)          # the FP32 path is 4M only
    assert e.value.status == tn.TN_ERR_UNSUPPORTED
    for prec in ("tf32", "bf16x3"):                         # 3M on the tensor cores
        assert tn.Plan(net, open_mask=om, precision=prec, complex_mult=3, trials=2).info()["n_steps"] > 0
    with pytest.raises(tn.TnError) as e:
        tn.Plan(net, open_mask=om, max_log2_intermediate=6)   # 12 open qubits > 2^6
    assert e.value.status == tn.TN_ERR_PLAN


def test_wire_counts(tn):
    circ, _, _ = rqcgen.config_circuit("c1")
    net = tn.Network(circ)
    gpq = net.gates_per_qubit()
    want = [int(np.sum((circ.gate_qubits[:, 0] == q) | (circ.gate_qubits[:, 1] == q)))
            for q in range(circ.n_qubits)]
    assert gpq == want


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_plan_respects_bound_and_reports(tn, name):
    cfg = rqcgen.CONFIGS[name]
    circ, om, _ = rqcgen.config_circuit(name)
    net = tn.Network(circ)
    plan = tn.Plan(net, open_mask=om, max_log2_intermediate=cfg["log2_bound"], trials=16)
    info = plan.info()
    assert info["n_open"] == cfg["k_open"]
    assert info["log2_max_intermediate"] <= cfg["log2_bound"]
    assert info["n_steps"] == info["n_leaves"] - 1
    assert sum(info["k_histogram"]) == info["n_steps"]
    shapes = plan.step_shapes()
    flops = sum(8 * 2 ** (m + k + n) for m, k, n, _ in shapes)
    assert math.isclose(flops, info["flops_per_slice"], rel_tol=1e-12)
    for m, k, n, _ in shapes:
        assert m + k <= cfg["log2_bound"] and k + n <= cfg["log2_bound"] and m + n <= cfg["log2_bound"]


def test_forced_slices_and_wire_labels(tn):
    circ, om, _ = rqcgen.config_circuit("c1")
    net = tn.Network(circ)
    gpq = net.gates_per_qubit()
    plan = tn.Plan(net, open_mask=om & 0xFF, max_log2_intermediate=30, min_log2_slices=5, trials=8)
    sl = plan.sliced_wires()
    assert len(sl) == 5 == plan.info()["log2_slices"]
    for q, t in sl:
        assert 0 <= q < circ.n_qubits and 1 <= t < gpq[q], "sliced wires are internal wires"
    assert len(set(sl)) == 5


def test_plan_is_deterministic(tn):
    circ, om, _ = rqcgen.config_circuit("c2")
    net = tn.Network(circ)
    a = tn.Plan(net, open_mask=om, max_log2_intermediate=22, trials=8, seed=3)
    b = tn.Plan(net, open_mask=om, max_log2_intermediate=22, trials=8, seed=3)
    assert a.step_shapes() == b.step_shapes() and a.sliced_wires() == b.sliced_wires()


def test_forced_slices_are_used_and_validated(tn):
    circ, om, _ = rqcgen.config_circuit("c1")
    net = tn.Network(circ)
    forced = [(0, 3), (5, 4), (9, 2), (2, 5)]
    plan = tn.Plan(net, open_mask=om & 0xF0F, max_log2_intermediate=30, forced_slices=forced, trials=8)
    sl = plan.sliced_wires()
    assert sl[:4] == forced
    assert plan.info()["log2_batch_slices"] == 0
    gpq = net.gates_per_qubit()
    for bad in ([(0, 0)], [(3, gpq[3])], [(99, 1)], [(0, 3), (0, 3)]):
        with pytest.raises(tn.TnError) as e:
            tn.Plan(net, open_mask=om, forced_slices=bad, trials=2)
        assert e.value.status == tn.TN_ERR_ARG


def test_mem_weight_option(tn):
    """The order search's memory weight is an option: validated, and a plan
    built with the default weight equals one built with weight 32 explicitly."""
    circ, om, _ = rqcgen.config_circuit("c2")
    net = tn.Network(circ)
    a = tn.Plan(net, open_mask=om, max_log2_intermediate=22, trials=8, seed=3)
    b = tn.Plan(net, open_mask=om, max_log2_intermediate=22, trials=8, seed=3, mem_weight=32.0)
    assert a.step_shapes() == b.step_shapes()
    tn.Plan(net, open_mask=om, max_log2_intermediate=22, trials=8, seed=3, mem_weight=2.0)
    with pytest.raises(tn.TnError) as e:
        tn.Plan(net, open_mask=om, max_log2_intermediate=22, trials=8, mem_weight=1e12)
    assert e.value.status == tn.TN_ERR_ARG


def test_sm_pairs_option(tn):
    """SM pairs are on by default, can be switched off, and nothing else is
    accepted; the order and slices do not depend on it (a kernel choice only)."""
    assert tn.default_opts().sm_pairs == 1
    circ, om, _ = rqcgen.config_circuit("c2")
    net = tn.Network(circ)
    a = tn.Plan(net, open_mask=om, max_log2_intermediate=22, trials=8, seed=3, precision="bf16x3")
    b = tn.Plan(net, open_mask=om, max_log2_intermediate=22, trials=8, seed=3, precision="bf16x3", sm_pairs=0)
    assert a.step_shapes() == b.step_shapes() and a.sliced_wires() == b.sliced_wires()
    for bad in (2, -1):
        with pytest.raises(tn.TnError) as e:
            tn.Plan(net, open_mask=om, max_log2_intermediate=22, trials=8, sm_pairs=bad)
        assert e.value.status == tn.TN_ERR_ARG


@pytest.mark.parametrize("name", ["c2", "c3"])
def test_layout_pass_guarantees(tn, name):
    """The planner stores every streamed operand A as [its contracted wires,
    its rows (free wires, then A-only batch bits)], shared batch bits on top,
    so tiles of A are plain row-major blocks; every operand's positions form a
    permutation; results that depend on no slice exist (reused prologue steps)
    and the root depends on the slices when the plan is sliced."""
    cfg = rqcgen.CONFIGS[name]
    circ, om, _ = rqcgen.config_circuit(name)
    plan = tn.Plan(tn.Network(circ), open_mask=om, max_log2_intermediate=cfg["log2_bound"],
                   min_log2_slices=cfg["log2_slices"], trials=16, precision="bf16x3")
    shapes = plan.step_shapes()
    flags = []
    for i, (m, k, n, b) in enumerate(shapes):
        L = plan.step_layout(i)
        assert L["a_k"] == list(range(k)), "contracted wires first in A"
        assert L["a_m"] == list(range(k, k + m)), "A's rows contiguous after them"
        assert all(p >= k + m for p in L["a_b"]), "shared batch bits on top of A"
        assert sorted(L["a_k"] + L["a_m"] + L["a_b"]) == list(range(k + m + b))
        assert sorted(L["b_k"] + L["b_n"] + L["b_b"]) == list(range(k + n + b))
        assert sorted(L["c_m"] + L["c_n"] + L["c_b"]) == list(range(m + n + b))
        flags.append(L["dep_flags"])
    assert set(flags) <= {0, 1, 2, 3}
    assert 0 in flags or 2 in flags
    if plan.info()["log2_slices"] > 0:
        assert flags[-1] & 1


def test_chunk_launches_needs_device_state(tn):
    circ, om, _ = rqcgen.config_circuit("c1")
    plan = tn.Plan(tn.Network(circ), open_mask=om, trials=2)
    with pytest.raises(tn.TnError) as e:
        plan.chunk_launches()
    assert e.value.status == tn.TN_ERR_ARG


def test_compute_calls_reject_bad_arguments_before_device_work(tn):
    """The compute entry points validate their host-side arguments first and
    return TN_ERR_ARG (TN_ERR_UNSUPPORTED for 3M on the FP32 path) with a
    message, before any device memory is touched or kernel launched; the device
    pointers below are never dereferenced."""
    import ctypes
    lib = tn.load()
    ERR, UNS = tn.TN_ERR_ARG, tn.TN_ERR_UNSUPPORTED
    dev = ctypes.c_void_p(1 << 20)   # stands for a device buffer
    x = ctypes.c_double()

    def i32(v):
        return (ctypes.c_int32 * max(1, len(v)))(*v)

    def expect(status, want):
        assert status == want
        assert lib.tn_last_error()

    # tn_xeb: NULL, empty, qubit count
    expect(lib.tn_xeb(None, 4, 10, ctypes.byref(x), None), ERR)
    expect(lib.tn_xeb(dev, 0, 10, ctypes.byref(x), None), ERR)
    expect(lib.tn_xeb(dev, 4, -1, ctypes.byref(x), None), ERR)
    # tn_frugal_sample: bound, empty batch, draw count
    first = (ctypes.c_int64 * 4)()
    for m_bound in (0.0, -1.0, float("nan"), float("inf")):
        expect(lib.tn_frugal_sample(dev, 64, 6, m_bound, dev, dev, 8, 4, first, None), ERR)
    expect(lib.tn_frugal_sample(dev, 0, 6, 10.0, dev, dev, 8, 4, first, None), ERR)
    expect(lib.tn_frugal_sample(dev, 64, 6, 10.0, dev, dev, 1 << 40, 4, first, None), ERR)
    # tn_permute: rank range, not a permutation, negative batch
    expect(lib.tn_permute(dev, dev, 35, i32(list(range(35))), 1, None), ERR)
    expect(lib.tn_permute(dev, dev, 3, i32([0, 0, 2]), 1, None), ERR)
    expect(lib.tn_permute(dev, dev, 3, i32([0, 3, 1]), 1, None), ERR)
    expect(lib.tn_permute(dev, dev, 3, i32([2, 1, 0]), -1, None), ERR)

    # tn_contract_pair: A(0,1,2) B(2,3) -> C(0,1,3) is valid; break one thing at a time
    def pair(aw, bw, cw, batch=1, prec=tn.PREC["fp32"], cm=4):
        return lib.tn_contract_pair(dev, i32(aw), len(aw), dev, i32(bw), len(bw), dev, i32(cw), len(cw),
                                    batch, prec, cm, None)
    expect(pair([0, 1, 1], [1, 3], [0, 3]), ERR)                    # repeated wire in A
    expect(pair([0, 1, 2], [2, 2], [0, 1]), ERR)                    # repeated wire in B
    expect(pair([0, 1, 2], [2, 3], [0, 1]), ERR)                    # C misses B's free wire
    expect(pair([0, 1, 2], [2, 3], [0, 3, 7]), ERR)                 # C has a foreign wire
    expect(pair([0, 1, 2], [2, 3], [0, 1, 3], batch=0), ERR)
    expect(pair([0, 1, 2], [2, 3], [0, 1, 3], prec=17), ERR)
    expect(pair([0, 1, 2], [2, 3], [0, 1, 3], cm=5), ERR)
    expect(pair([0, 1, 2], [2, 3], [0, 1, 3], cm=3), UNS)           # 3M needs a tensor-core mode

    # tn_contract_slices: NULL, no batch, slice range beyond 2^S (S = 5 here)
    circ, om, _ = rqcgen.config_circuit("c1")
    plan = tn.Plan(tn.Network(circ), open_mask=om & 0xFF, max_log2_intermediate=30, min_log2_slices=5, trials=4)
    bits = (ctypes.c_uint64 * 1)(0)
    expect(lib.tn_contract_slices(plan.handle, 0, 32, None, 1, dev, None), ERR)
    expect(lib.tn_contract_slices(plan.handle, 0, 32, bits, 0, dev, None), ERR)
    expect(lib.tn_contract_slices(plan.handle, 30, 3, bits, 1, dev, None), ERR)
    expect(lib.tn_contract_slices(plan.handle, 33, 0, bits, 1, dev, None), ERR)
    assert lib.tn_contract_slices(plan.handle, 32, 0, bits, 1, dev, None) == tn.TN_OK   # empty range: no work

    # tn_plan_select: candidate count
    o = tn.default_opts()
    h = ctypes.c_void_p()
    expect(lib.tn_plan_select(tn.Network(circ).handle, ctypes.byref(o), 0, 0, None, ctypes.byref(h), None), ERR)


def test_model_time_is_the_roofline_sum_over_chunk_steps(tn):
    """tn_plan_model_time = sum over the steps that run every chunk (result
    depends on the slice id) of max(8 m k n 2^b / P, 8 (|A|+|B|+|C|) / BW), with
    |A| = 2^(m+k+b), |B| = 2^(k+n+b), |C| = 2^(m+n+b) from the step shapes; it
    grows when either peak shrinks and rejects non-positive peaks."""
    cfg = rqcgen.CONFIGS["c3"]
    circ, om, _ = rqcgen.config_circuit("c3")
    plan = tn.Plan(tn.Network(circ), open_mask=om, max_log2_intermediate=cfg["log2_bound"],
                   min_log2_slices=cfg["log2_slices"], trials=16, precision="bf16x3")
    P, BW = 639.8e12, 6783.5e9
    want = 0.0
    for i, (m, k, n, b) in enumerate(plan.step_shapes()):
        if plan.step_layout(i)["dep_flags"] & 1:
            want += max(8.0 * 2 ** (m + k + n + b) / P,
                        8.0 * (2 ** (m + k + b) + 2 ** (k + n + b) + 2 ** (m + n + b)) / BW)
    got = plan.model_time(P, BW)
    assert got == pytest.approx(want, rel=1e-12) and got > 0
    assert plan.model_time(P / 2, BW) >= got and plan.model_time(P, BW / 2) >= got
    assert plan.model_time(P / 2, BW / 2) == pytest.approx(2 * got, rel=1e-12)
    for bad in ((0.0, BW), (P, -1.0), (float("nan"), BW)):
        with pytest.raises(tn.TnError) as e:
            plan.model_time(*bad)
        assert e.value.status == tn.TN_ERR_ARG


def test_plan_rank_models_every_candidate(tn):
    """tn_plan_rank gives each (seed, memory weight) candidate the modeled time
    of one batch of the plan tn_plan builds from the same options: the chunk's
    tn_plan_model_time x 2^(S - b) plus the roofline sum over the steps that
    run once per batch (dependence flags 2); a candidate that cannot be planned
    (no batch fits the arena cap) gets -1, and a pool where none can is
    TN_ERR_PLAN."""
    circ, om, _ = rqcgen.config_circuit("c2")
    net = tn.Network(circ)
    kw = dict(open_mask=om, max_log2_intermediate=22, min_log2_slices=4, trials=8, precision="bf16x3")
    P, BW = 631.6e12, 6786.9e9
    seeds, weights = [3, 4, 3], [32.0, 8.0, 128.0]
    got = tn.rank_plans(net, seeds, weights, P, BW, **kw)
    for s, w, g in zip(seeds, weights, got):
        p = tn.Plan(net, seed=s, mem_weight=w, **kw)
        i = p.info()
        per_batch = 0.0
        for j, (m, k, n, b) in enumerate(p.step_shapes()):
            if p.step_layout(j)["dep_flags"] == 2:
                per_batch += max(8.0 * 2 ** (m + k + n + b) / P,
                                 8.0 * (2 ** (m + k + b) + 2 ** (k + n + b) + 2 ** (m + n + b)) / BW)
        assert per_batch > 0
        want = p.model_time(P, BW) * 2.0 ** (i["log2_slices"] - i["log2_batch_slices"]) + per_batch
        assert g == pytest.approx(want, rel=1e-12) and g > 0
    with pytest.raises(tn.TnError) as e:
        tn.rank_plans(net, [1], [32.0], P, BW, max_arena_bytes=1 << 10, **kw)
    assert e.value.status == tn.TN_ERR_PLAN
    with pytest.raises(tn.TnError) as e:
        tn.rank_plans(net, [1], [1e12], P, BW, **kw)
    assert e.value.status == tn.TN_ERR_ARG
    with pytest.raises(tn.TnError) as e:
        tn.rank_plans(net, [1], [32.0], 0.0, BW, **kw)
    assert e.value.status == tn.TN_ERR_ARG


def test_pool_ranking_is_sorted_and_reproducible(tn):
    """The pool helper plans the seed x weight grid, drops nothing that
    planned, sorts by modeled time, and gives the same ranking twice."""
    from paper_2111_01066_gb300 import pool
    circ, om, _ = rqcgen.config_circuit("c2")
    net = tn.Network(circ)
    kw = dict(open_mask=om, max_log2_intermediate=22, trials=4)
    assert pool.candidate_grid(5) == [(1, 8.0), (1, 32.0), (1, 128.0), (2, 8.0), (2, 32.0)]
    a = pool.rank_pool(net, 6, "bf16x3", 4, **kw)
    b = pool.rank_pool(net, 6, "bf16x3", 4, **kw)
    assert a == b and len(a) == 6
    assert [r["model_seconds"] for r in a] == sorted(r["model_seconds"] for r in a)
    assert {(r["seed"], r["mem_weight"]) for r in a} == set(pool.candidate_grid(6))


@pytest.mark.parametrize("name", ["c1", "c3"])
def test_plan_tree_is_a_complete_tree_over_the_circuit(tn, name):
    """tn_plan_tree: every gate sits in exactly one leaf, every leaf holds a
    gate, and the steps merge every node exactly once into one root; each
    step's operands are the nodes whose wires its layout reads (leaf or earlier
    step), so the tree is the one the executor runs."""
    cfg = rqcgen.CONFIGS[name]
    circ, om, _ = rqcgen.config_circuit(name)
    plan = tn.Plan(tn.Network(circ), open_mask=om, max_log2_intermediate=cfg["log2_bound"],
                   min_log2_slices=cfg["log2_slices"], trials=8)
    leaf_of_gate, nodes = plan.tree(circ.n_gates)
    n_leaves = plan.info()["n_leaves"]
    assert sorted(set(leaf_of_gate)) == list(range(n_leaves))
    assert len(nodes) == n_leaves - 1 == plan.info()["n_steps"]
    alive = set(range(n_leaves))
    for j, (x, y) in enumerate(nodes):
        assert x in alive and y in alive and x != y
        alive -= {x, y}
        alive.add(n_leaves + j)
    assert alive == {2 * n_leaves - 2}
    with pytest.raises(tn.TnError):
        plan.tree(circ.n_gates - 1)


def test_select_list_and_device_sync_validate_before_device_work(tn):
    import ctypes
    lib = tn.load()
    circ, om, _ = rqcgen.config_circuit("c1")
    net = tn.Network(circ)
    o = tn.default_opts()
    h = ctypes.c_void_p()
    seeds = (ctypes.c_uint64 * 2)(1, 2)
    w = (ctypes.c_double * 2)(32.0, 8.0)
    bad_w = (ctypes.c_double * 2)(32.0, 1e12)
    assert lib.tn_plan_select_list(net.handle, ctypes.byref(o), 0, seeds, w, 0, None, ctypes.byref(h),
                                   None) == tn.TN_ERR_ARG
    assert lib.tn_plan_select_list(net.handle, ctypes.byref(o), 2, None, w, 0, None, ctypes.byref(h),
                                   None) == tn.TN_ERR_ARG
    assert lib.tn_plan_select_list(net.handle, ctypes.byref(o), 2, seeds, bad_w, 0, None, ctypes.byref(h),
                                   None) == tn.TN_ERR_ARG
    plan = tn.Plan(net, open_mask=om, trials=2)
    with pytest.raises(tn.TnError) as e:
        plan.batch_launches()
    assert e.value.status == tn.TN_ERR_ARG


def test_tuning_calls_validate_before_device_work(tn):
    """tn_plan_get_tuning / tn_plan_set_tuning need the plan's device state (one
    contract call) and reject NULL arguments, short buffers and wrong lengths
    before touching anything."""
    import ctypes
    lib = tn.load()
    circ, om, _ = rqcgen.config_circuit("c1")
    plan = tn.Plan(tn.Network(circ), open_mask=om, trials=2)
    n = plan.info()["n_steps"]
    buf = (ctypes.c_int32 * (n * tn.TN_TUNING_INTS))()
    cnt = ctypes.c_int32()
    for args in ((plan.handle, None, len(buf), ctypes.byref(cnt)), (plan.handle, buf, len(buf), None),
                 (None, buf, len(buf), ctypes.byref(cnt)), (plan.handle, buf, len(buf), ctypes.byref(cnt))):
        assert lib.tn_plan_get_tuning(*args) == tn.TN_ERR_ARG   # the last: no device state yet
    for args in ((plan.handle, None, len(buf)), (None, buf, len(buf)), (plan.handle, buf, len(buf))):
        assert lib.tn_plan_set_tuning(*args) == tn.TN_ERR_ARG
    with pytest.raises(tn.TnError) as e:
        plan.get_tuning()
    assert e.value.status == tn.TN_ERR_ARG


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_step_groups_are_consecutive_independent_and_small(tn, name):
    """Small steps come in groups that the executor runs as one launch: a
    group's steps are consecutive, of one dependence class (per batch or per
    chunk), read no result of another step of the group, and are under 2^20
    multiply-adds; steps run once per plan, then once per batch, then per chunk."""
    cfg = rqcgen.CONFIGS[name]
    circ, om, _ = rqcgen.config_circuit(name)
    plan = tn.Plan(tn.Network(circ), open_mask=om, max_log2_intermediate=cfg["log2_bound"],
                   min_log2_slices=max(cfg["log2_slices"], 3), trials=16, precision="bf16x3")
    n = plan.info()["n_steps"]
    n_leaves = plan.info()["n_leaves"]
    _, nodes = plan.tree(circ.n_gates)
    lay = [plan.step_layout(i) for i in range(n)]
    shapes = plan.step_shapes()
    cls = [0 if l["dep_flags"] == 0 else (1 if l["dep_flags"] == 2 else 2) for l in lay]
    assert cls == sorted(cls), "once per plan, then once per batch, then per chunk"
    groups = {}
    for i, l in enumerate(lay):
        if l["group"] >= 0:
            groups.setdefault(l["group"], []).append(i)
    assert groups
    for g, members in groups.items():
        assert members == list(range(members[0], members[-1] + 1))
        for i in members:
            assert (lay[i]["dep_flags"] == 2) == (lay[members[0]]["dep_flags"] == 2) and lay[i]["dep_flags"] > 0
            assert sum(shapes[i]) < 20
            for x in nodes[i]:
                assert x - n_leaves not in members or x < n_leaves
