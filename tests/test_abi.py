"""The C-ABI library builds, loads and exports every entry point declared in include/sg.h, and
its host-side logic (argument checking, instance validation, layout sizing) works without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1906_11195_gb300 as sg
import sg_inputs
from paper_1906_11195_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ctypes.CDLL(_build.LIB)


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(sg.EXPORTED)


def _graph(n=200, c=4.0, seed=3):
    rp, col, eid = sg_inputs.poisson_graph(n, c, seed)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, seed)
    return dict(row_ptr=rp, col=col, jbits=jb, seed=5, temps=[1.0, 1.0])


def test_create_and_size_without_gpu(lib):
    g = _graph()
    for kernel in (sg.SG_VB_PLAIN, sg.SG_VB_PACKED):
        h = sg.sg_create_vb([g], 8, 2, kernel, [0, 4], [0, 4, 8])
        assert sg.sg_workspace_bytes(h) > 0
        assert sg.sg_result_shape(h) == (1, 2, 8, 2, 3)
        thr = sg.sg_get_thresholds(h, 2 * 64)
        assert thr[0] == 0xFFFFFFFF and thr[1] == int(np.floor(2.0**32 * np.exp(-2.0)))
        with pytest.raises(sg.SGError) as e:
            sg.sg_sweep(h, 1)
        assert e.value.code == sg.SG_ESTATE
        sg.sg_destroy(h)


@pytest.mark.parametrize("defect", ["asymmetric", "self_loop", "duplicate", "coupling_mismatch",
                                    "degree", "bad_schedule", "bad_replicas", "bad_temp"])
def test_invalid_instances_are_rejected(lib, defect):
    g = _graph()
    tw, tm, R, kernel = [0], [0, 1], 2, sg.SG_VB_PACKED
    rp, col, jb = g["row_ptr"].copy(), g["col"].copy(), g["jbits"].copy()
    if defect == "asymmetric":
        col[0] = (col[0] + 1) % 200 if (col[0] + 1) % 200 != 0 else 2
    elif defect == "self_loop":
        col[rp[5]] = 5
    elif defect == "duplicate":
        col[rp[7] + 1] = col[rp[7]]
    elif defect == "coupling_mismatch":
        jb[0] ^= np.uint64(1)
    elif defect == "degree":
        n = 70
        ei = np.zeros(n - 1, dtype=np.int64)
        ej = np.arange(1, n)
        rp, col, _ = sg_inputs.csr_from_edges(n, ei, ej)
        jb = np.zeros(col.size, dtype=np.uint64)
    elif defect == "bad_schedule":
        tw = [4, 2]
    elif defect == "bad_replicas":
        R = 3
    elif defect == "bad_temp":
        g["temps"] = [-1.0, 1.0]
    g2 = dict(g, row_ptr=rp, col=col, jbits=jb)
    with pytest.raises(sg.SGError) as e:
        sg.sg_create_vb([g2], 64, R, kernel, tw, tm)
    assert e.value.code == sg.SG_EINVAL
    assert sg.sg_last_error()


def test_schedule_helper():
    tw, tm = sg_inputs.log_schedule([0, 1, 4], 10)
    assert list(tw) == [0, 1, 4]
    assert list(tm) == [0, 1, 2, 3, 4, 5, 6, 8, 9]


def test_sk_create_and_validation_without_gpu(lib):
    J = sg_inputs.sk_couplings(300, 1)
    h = sg.sg_create_sk(J, 32, [0.4] * 32, 7, sg.SG_SK_BLOCKED, 128, [0, 3], [0, 3, 5])
    assert sg.sg_workspace_bytes(h) > 384 * 384
    assert sg.sg_result_shape(h) == (1, 32, 1, 2, 3)
    thr = sg.sg_get_thresholds(h, 32 * 300).reshape(32, 300)
    assert thr[0, 0] == 0xFFFFFFFF
    assert thr[0, 1] == int(np.floor(2.0**32 * np.exp(-(2.0 / 0.4) / np.sqrt(300))))
    sg.sg_destroy(h)
    bad = J.copy()
    bad[0, 1] = -bad[0, 1]
    for args in [(bad, 32, sg.SG_SK_BLOCKED, 128),      # asymmetric
                 (J, 20, sg.SG_SK_BLOCKED, 128),        # replicas not a multiple of 16
                 (J, 32, sg.SG_SK_BLOCKED, 96),         # unsupported block
                 (np.eye(300, dtype=np.int8), 32, sg.SG_SK_PLAIN, 0)]:  # nonzero diagonal
        with pytest.raises(sg.SGError) as e:
            sg.sg_create_sk(args[0], args[1], [0.4] * args[1], 1, args[2], args[3], [], [])
        assert e.value.code == sg.SG_EINVAL


def test_size_limits_are_rejected_before_any_array_is_read(lib):
    """n outside [2, SG_VB_MAX_N] (VB) or [2, 32768] (SK), no graphs, too many lanes: SG_EINVAL,
    decided from the sizes alone (the arrays passed are far too small to be read)."""
    import ctypes
    L = sg._load()
    tiny_i = np.zeros(4, dtype=np.int32)
    tiny_u = np.zeros(4, dtype=np.uint64)
    temps = np.ones(2, dtype=np.float64)
    h = ctypes.c_void_p()
    for n in (0, 1, (1 << 26), (1 << 26) + 5):
        g = (sg.sg_vb_graph * 1)()
        g[0] = sg.sg_vb_graph(n, tiny_i.ctypes.data, tiny_i.ctypes.data, tiny_u.ctypes.data, 1,
                              temps.ctypes.data)
        rc = L.sg_create_vb(ctypes.cast(g, ctypes.c_void_p), 1, 64, 2, sg.SG_VB_PACKED, None, 0,
                            None, 0, ctypes.byref(h))
        assert rc == sg.SG_EINVAL, n
    g = (sg.sg_vb_graph * 1)()
    g[0] = sg.sg_vb_graph(2, tiny_i.ctypes.data, tiny_i.ctypes.data, tiny_u.ctypes.data, 1,
                          temps.ctypes.data)
    for n_graphs, lanes in ((0, 64), (1, 0), (1, 65)):
        rc = L.sg_create_vb(ctypes.cast(g, ctypes.c_void_p), n_graphs, lanes, 2, sg.SG_VB_PACKED,
                            None, 0, None, 0, ctypes.byref(h))
        assert rc == sg.SG_EINVAL, (n_graphs, lanes)
    tiny_j = np.zeros(4, dtype=np.int8)
    for n in (0, 1, 32769):
        rc = L.sg_create_sk(n, tiny_j.ctypes.data, 16, temps.ctypes.data, 1, sg.SG_SK_BLOCKED, 128,
                            None, 0, None, 0, ctypes.byref(h))
        assert rc == sg.SG_EINVAL, n
    assert sg.sg_last_error()


def test_edgeless_graph_is_accepted(lib):
    """A graph with no edges at all (every vertex isolated) is a valid, degenerate instance."""
    n = 1000
    rp = np.zeros(n + 1, dtype=np.int32)
    g = dict(row_ptr=rp, col=np.zeros(0, dtype=np.int32), jbits=np.zeros(0, dtype=np.uint64),
             seed=3, temps=[1.0, 0.5])
    for kernel in (sg.SG_VB_PLAIN, sg.SG_VB_PACKED):
        h = sg.sg_create_vb([g], 64, 2, kernel, [0], [0, 1, 2])
        assert sg.sg_workspace_bytes(h) > 0
        sg.sg_destroy(h)


def test_windows_are_validated_and_grow_the_workspace(lib):
    g = _graph()
    h = sg.sg_create_vb([g], 64, 2, sg.SG_VB_PACKED, [0, 4], [0, 4, 8])
    base = sg.sg_workspace_bytes(h)
    for bad in ([5], [4, 4], [6, 3], [-1, 2]):
        with pytest.raises(sg.SGError) as e:
            sg.sg_set_windows(h, bad)
        assert e.value.code == sg.SG_EINVAL
    sg.sg_set_windows(h, sg_inputs.geometric_windows(2, 1000))
    assert sg.sg_workspace_bytes(h) > base
    with pytest.raises(sg.SGError) as e:  # nothing attached: no sums to read
        sg.sg_read_windows(h, 3)
    assert e.value.code == sg.SG_ESTATE
    sg.sg_destroy(h)


def test_undersized_workspace_is_rejected_before_use(lib):
    """sg_attach checks the size first: a workspace one byte short is SG_ENOMEM, and the pointer
    is never dereferenced (a dummy address suffices on a machine without a GPU)."""
    g = _graph()
    h = sg.sg_create_vb([g], 64, 2, sg.SG_VB_PACKED, [0], [0, 1])
    need = sg.sg_workspace_bytes(h)
    with pytest.raises(sg.SGError) as e:
        sg.sg_attach(h, 1 << 20, need - 1, 0)
    assert e.value.code == sg.SG_ENOMEM
    sg.sg_destroy(h)


def test_set_schedule_before_attach_resizes_the_workspace(lib):
    """sg_set_schedule before sg_attach: any valid schedule, the workspace follows its sizes;
    invalid arrays are SG_EINVAL and leave the handle's schedule as it was."""
    g = _graph()
    for kernel in (sg.SG_VB_PLAIN, sg.SG_VB_PACKED):
        h = sg.sg_create_vb([g], 8, 2, kernel, [0], [0, 1])
        base = sg.sg_workspace_bytes(h)
        sg.sg_set_schedule(h, [0, 4, 16], [0, 4, 8, 16, 20, 32])
        assert sg.sg_result_shape(h) == (1, 2, 8, 3, 6)
        assert sg.sg_workspace_bytes(h) > base
        for tw, tm in (([4, 2], [5]), ([0], [-1, 3]), ([1 << 32], [1]), ([0], [3, 3])):
            with pytest.raises(sg.SGError) as e:
                sg.sg_set_schedule(h, tw, tm)
            assert e.value.code == sg.SG_EINVAL
        assert sg.sg_result_shape(h) == (1, 2, 8, 3, 6)
        sg.sg_set_schedule(h, [], [])
        assert sg.sg_result_shape(h) == (1, 2, 8, 0, 0)
        assert sg.sg_workspace_bytes(h) < base
        sg.sg_destroy(h)
    J = sg_inputs.sk_couplings(200, 2)
    h = sg.sg_create_sk(J, 16, [0.4] * 16, 7, sg.SG_SK_BLOCKED, 128, [0], [0])
    base = sg.sg_workspace_bytes(h)
    sg.sg_set_schedule(h, [0, 3], [0, 3, 9])
    assert sg.sg_result_shape(h) == (1, 16, 1, 2, 3)
    assert sg.sg_workspace_bytes(h) > base
    sg.sg_destroy(h)
    samples = [dict(J=sg_inputs.sk_couplings(n, 3 + n), seed=n, temps=[0.5] * 16) for n in (100, 140)]
    h = sg.sg_create_sk_batch(samples, 16, sg.SG_SK_BLOCKED, 64, [0], [0])
    base = sg.sg_workspace_bytes(h)
    sg.sg_set_schedule(h, [0, 2, 5], [0, 2, 5, 7])
    assert sg.sg_result_shape(h) == (2, 16, 1, 3, 4)
    assert sg.sg_workspace_bytes(h) > base
    sg.sg_destroy(h)


def test_noalloc_rejects_host_pointers_before_launching(lib):
    """The allocation-free field call checks its pointers on the host: host memory (or memory of
    another device) is SG_EINVAL and nothing is launched; sizes beyond the static array too."""
    L = sg._load()
    J = np.zeros(64 * 64, dtype=np.int8)
    s = np.ones(16 * 64, dtype=np.int8)
    h = np.zeros(16 * 64, dtype=np.int32)
    for n, R in ((64, 16), (4096, 16), (64, 256), (64, 24), (1, 16)):
        rc = L.sg_sk_fields_noalloc(J.ctypes.data, s.ctypes.data, n, R, h.ctypes.data, None)
        assert rc == sg.SG_EINVAL, (n, R)
        assert sg.sg_last_error()


def test_transfer_bytes_start_at_zero(lib):
    g = _graph()
    h = sg.sg_create_vb([g], 64, 2, sg.SG_VB_PACKED, [0], [0, 1])
    assert sg.sg_transfer_bytes(h) == (0, 0)
    sg.sg_destroy(h)


def test_blocked_sk_schedule_is_validated(lib):
    cnt = ctypes.c_int32(0)
    for n, block in ((1, 128), (40000, 128), (1024, 100), (1024, 0)):
        assert lib.sg_sk_blocked_schedule(n, block, None, 0, ctypes.byref(cnt)) == sg.SG_EINVAL
    # capacity query, then a buffer one operation short
    assert lib.sg_sk_blocked_schedule(1024, 256, None, 0, ctypes.byref(cnt)) == sg.SG_EINVAL
    need = cnt.value
    assert need == len(sg.sg_sk_blocked_schedule(1024, 256)) > 0
    buf = (ctypes.c_int32 * (6 * need))()
    assert lib.sg_sk_blocked_schedule(1024, 256, buf, need - 1, ctypes.byref(cnt)) == sg.SG_EINVAL
    assert lib.sg_sk_blocked_schedule(1024, 256, buf, need, ctypes.byref(cnt)) == sg.SG_OK
    ops = np.frombuffer(buf, dtype=np.int32).reshape(need, 6)
    assert ops[0, 0] == 0 and set(ops[:, 0]) <= {0, 1, 2, 3, 4, 5}
    assert (ops[ops[:, 0] == 1, 2] == np.arange(4)).all()  # in-block kernels of blocks 0..3 in order


@pytest.mark.parametrize("n,c,seed", [(37, 3.0, 1), (5000, 4.0, 2), (200000, 4.0, 7)])
def test_library_colouring_equals_the_oracles(lib, n, c, seed):
    """The update order, checked on the host: the library's own greedy colouring and recolouring
    pass give every vertex the oracle's class (both written separately), for each graph of a
    batch; the bipartite regular graph keeps its two halves."""
    import oracle
    oracle.build()
    graphs = []
    for k, (nn, cc, sd) in enumerate([(n, c, seed), (n // 2 + 3, c, seed + 1)]):
        rp, col, eid = sg_inputs.poisson_graph(nn, cc, sd)
        jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, sd)
        graphs.append(dict(row_ptr=rp, col=col, jbits=jb, seed=k, temps=[1.0, 1.0]))
    h = sg.sg_create_vb(graphs, 64, 2, sg.SG_VB_PACKED, [0], [1])
    try:
        for b, g in enumerate(graphs):
            got, nc = sg.sg_vb_colouring(h, b, len(g["row_ptr"]) - 1)
            want, wnc = oracle.vb_colouring(g["row_ptr"], g["col"])
            assert nc == wnc and np.array_equal(got, want)
        with pytest.raises(sg.SGError):
            sg.sg_vb_colouring(h, 2, 10)
    finally:
        sg.sg_destroy(h)
    rp, col, eid = sg_inputs.random_regular_graph(1000, 4, 3, bipartite=True)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, 3)
    h = sg.sg_create_vb([dict(row_ptr=rp, col=col, jbits=jb, seed=1, temps=[1.0, 1.0])], 64, 2,
                        sg.SG_VB_PACKED, [0], [1])
    try:
        got, nc = sg.sg_vb_colouring(h, 0, 1000)
        assert nc == 2 and np.array_equal(got, (np.arange(1000) < 500).astype(np.int32))
    finally:
        sg.sg_destroy(h)


def test_library_thresholds_equal_the_oracles_on_the_host(lib):
    """The Metropolis threshold tables (integer thresholds floor(2^32 exp(-dE/T)) in double
    precision), computed by the library at creation, equal the oracle's: VB per replica for every
    degree up to the limit, SK per replica for every k, at finite, zero and infinite T."""
    import math

    import oracle
    oracle.build()
    rp, col, eid = sg_inputs.poisson_graph(300, 4.0, 9)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, 9)
    temps = [1.0, 0.6, 0.0, math.inf]
    h = sg.sg_create_vb([dict(row_ptr=rp, col=col, jbits=jb, seed=1, temps=temps)], 64, 4,
                        sg.SG_VB_PACKED, [0], [1])
    try:
        thr = sg.sg_get_thresholds(h, 4 * 64).reshape(4, 64)
        for r, T in enumerate(temps):
            assert np.array_equal(thr[r], oracle.vb_thresholds(T, 63))
    finally:
        sg.sg_destroy(h)
    n = 300
    J = sg_inputs.sk_couplings(n, 4)
    stemps = [0.4] * 8 + [0.6] * 8
    h = sg.sg_create_sk(J, 16, stemps, 1, sg.SG_SK_BLOCKED, 128, [0], [1])
    try:
        thr = sg.sg_get_thresholds(h, 16 * n).reshape(16, n)
        assert np.array_equal(thr[0], oracle.sk_thresholds(0.4, n))
        assert np.array_equal(thr[15], oracle.sk_thresholds(0.6, n))
    finally:
        sg.sg_destroy(h)
