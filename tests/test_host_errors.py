"""Host-side error behaviour of the C ABI (include/lbdd.h), on the CPU.

Every call validates its arguments before it touches the device, so invalid
arguments return LBDD_ERR_ARG and leave the output handle NULL on any
machine.  Valid arguments on a machine without a compute-capability-10.3
GPU fail with LBDD_ERR_CUDA or LBDD_ERR_NODEV: there is no CPU fallback,
and the Python binding raises.  The no-device cases skip when a GPU is
present (they would then run real work on placeholder data).
"""
import ctypes

import numpy as np
import pytest

import lbdd_inputs as L


@pytest.fixture(scope="module")
def lb():
    import paper_2304_06543_gb300 as lb
    lb.load()
    return lb


@pytest.fixture(scope="module")
def lib(lb):
    return lb.load()


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _gpu_present():
    import torch
    return torch.cuda.is_available()


no_gpu = pytest.mark.skipif("_gpu_present()", reason="a GPU is present")


def test_create_rejects_bad_arguments(lb, lib):
    n, k = 8, 3
    cm = np.ones((n, k), np.int32)
    cap = np.full(k, 2, np.int32)
    pen = np.full(k, 5, np.int32)
    h = ctypes.c_void_p()

    def create(n=n, k=k, cm=cm, dtype=lb.CM_I32, cap=cap, pen=pen):
        h.value = None
        rc = lib.lbdd_create(ctypes.byref(h), n, k, None if cm is None else _ptr(cm), dtype, 0,
                             None if cap is None else _ptr(cap),
                             None if pen is None else _ptr(pen), None)
        assert h.value is None
        return rc

    assert create(n=0) == lb.ERR_ARG
    assert create(k=0) == lb.ERR_ARG
    assert create(k=65536) == lb.ERR_ARG           # node ids are packed in 16 bits
    kmax = lib.lbdd_max_centers()
    wide = np.ones((2, kmax + 1), np.int32)
    ones = np.ones(kmax + 1, np.int32)
    h.value = None
    assert lib.lbdd_create(ctypes.byref(h), 2, kmax + 1, _ptr(wide), lb.CM_I32, 0, _ptr(ones),
                           _ptr(ones), None) == lb.ERR_ARG   # before any device work
    assert h.value is None
    assert create(dtype=7) == lb.ERR_ARG
    assert create(cm=None) == lb.ERR_ARG
    assert create(cap=None) == lb.ERR_ARG
    assert create(pen=None) == lb.ERR_ARG
    for bad in (0, -1):
        c = cap.copy()
        c[1] = bad
        assert create(cap=c) == lb.ERR_ARG           # capacities are positive
        p = pen.copy()
        p[2] = bad
        assert create(pen=p) == lb.ERR_ARG           # Def. 4: penalties are positive
    assert lib.lbdd_create(None, n, k, _ptr(cm), lb.CM_I32, 0, _ptr(cap), _ptr(pen),
                           None) == lb.ERR_ARG


def test_create_strict_rejects_bad_arguments(lb, lib):
    n, k = 8, 3
    cm = np.ones((n, k), np.int32)
    cap = np.full(k, 2, np.int32)
    h = ctypes.c_void_p()
    # k + 1 centers with the dummy one must still fit 16-bit node ids
    assert lib.lbdd_create_strict(ctypes.byref(h), n, 65535, _ptr(cm), lb.CM_I32, 0, _ptr(cap),
                                  None) == lb.ERR_ARG
    assert lib.lbdd_create_strict(ctypes.byref(h), n, k, _ptr(cm), 3, 0, _ptr(cap),
                                  None) == lb.ERR_ARG
    c = cap.copy()
    c[0] = 0
    assert lib.lbdd_create_strict(ctypes.byref(h), n, k, _ptr(cm), lb.CM_I32, 0, _ptr(c),
                                  None) == lb.ERR_ARG
    # k = the limit, capacities short of n: the dummy center makes k + 1
    kmax = lib.lbdd_max_centers()
    wide = np.ones((kmax + 1, kmax), np.int32)
    ones = np.ones(kmax, np.int32)
    assert lib.lbdd_create_strict(ctypes.byref(h), kmax + 1, kmax, _ptr(wide), lb.CM_I32, 0,
                                  _ptr(ones), None) == lb.ERR_ARG
    assert h.value is None


def test_null_handles_are_rejected(lb, lib):
    i64 = ctypes.c_int64()
    buf = np.zeros(16, np.int32)
    assert lib.lbdd_solve(None, -1) == lb.ERR_ARG
    assert lib.lbdd_reset(None) == lb.ERR_ARG
    u = ctypes.c_int32()
    assert lib.lbdd_insert(None, _ptr(buf), lb.CM_I32, ctypes.byref(u)) == lb.ERR_ARG
    assert lib.lbdd_set_option(None, lb.OPT_CLUSTER, 1) == lb.ERR_ARG
    assert lib.lbdd_set_penalty_table(None, _ptr(buf), 1) == lb.ERR_ARG
    assert lib.lbdd_objective(None, ctypes.byref(i64)) == lb.ERR_ARG
    assert lib.lbdd_rounds_done(None, ctypes.byref(i64)) == lb.ERR_ARG
    assert lib.lbdd_assignment(None, _ptr(buf), 0) == lb.ERR_ARG
    assert lib.lbdd_loads(None, _ptr(buf)) == lb.ERR_ARG
    assert lib.lbdd_best_transfer_table(None, _ptr(buf), _ptr(buf), 0) == lb.ERR_ARG
    assert lib.lbdd_batch_run(None, -1) == lb.ERR_ARG
    assert lib.lbdd_batch_plan(None, None, None, None, None, None, 0) == lb.ERR_ARG
    assert lib.lbdd_solve_batch(None, 1, -1, 0, 0, None) == lb.ERR_ARG
    assert lib.lbdd_autotune(None, 1, 64, None) == lb.ERR_ARG
    b = ctypes.c_void_p(1)
    assert lib.lbdd_batch_create(ctypes.byref(b), None, 1, 0, 0, None) == lb.ERR_ARG
    assert b.value is None
    assert lib.lbdd_server_submit(None, 1, 1, _ptr(buf), 0, _ptr(buf), _ptr(buf), _ptr(buf),
                                  ctypes.byref(i64)) == lb.ERR_ARG
    assert lib.lbdd_server_poll(None, 1, 0, None) == lb.ERR_ARG
    assert lib.lbdd_server_release(None, 1) == lb.ERR_ARG
    assert lib.lbdd_server_get_stats(None, None) == lb.ERR_ARG
    # destroy calls accept NULL
    lib.lbdd_destroy(None)
    lib.lbdd_batch_destroy(None)
    lib.lbdd_server_destroy(None)


def test_server_config_is_validated(lb, lib):
    s = ctypes.c_void_p(1)
    for budget, max_active, quantum, cluster in [(0, 0, 0, 0), (1 << 30, -1, 0, 0),
                                                 (1 << 30, 0, -5, 0), (1 << 30, 0, 0, 3),
                                                 (1 << 30, 0, 0, 32)]:
        cfg = lb._ServerConfig(budget, max_active, quantum, cluster)
        assert lib.lbdd_server_create(ctypes.byref(s), ctypes.byref(cfg)) == lb.ERR_ARG
        assert s.value is None
    assert lib.lbdd_server_create(ctypes.byref(s), None) == lb.ERR_ARG


def test_scan_and_road_arguments_are_validated(lb, lib):
    ws = lib.lbdd_best_transfer_workspace(100, 10)
    assert ws > 0
    a16 = ctypes.c_void_p(1 << 20)      # never dereferenced: every case below is invalid
    odd = ctypes.c_void_p((1 << 20) + 4)

    def bt(n=100, k=10, cm=a16, dtype=lb.CM_I32, ld=12, ws_bytes=ws):
        return lib.lbdd_best_transfer(n, k, cm, dtype, ld, a16, a16, a16, a16, ws_bytes, None)

    assert bt(n=0) == lb.ERR_ARG
    assert bt(k=0) == lb.ERR_ARG
    assert bt(dtype=9) == lb.ERR_ARG
    assert bt(ld=9) == lb.ERR_ARG                 # pitch below k
    assert bt(ld=10) == lb.ERR_ARG                # 40-byte rows: not a 16-byte multiple
    assert bt(cm=odd) == lb.ERR_ARG               # CM base not 16-byte aligned
    assert bt(ws_bytes=ws - 1) == lb.ERR_ARG      # workspace too small
    assert lib.lbdd_best_transfer_noalloc(ctypes.c_int32(0), ctypes.c_int32(10), a16,
                                          ctypes.c_int(lb.CM_I32), ctypes.c_int64(12), a16,
                                          a16, a16, None) == lb.ERR_ARG
    # road CM: sizes and null pointers
    assert lib.lbdd_road_cm(0, a16, a16, a16, 1, a16, 1, a16, a16, 1, None) == lb.ERR_ARG
    assert lib.lbdd_road_cm(4, a16, a16, a16, 2, a16, 1, a16, a16, 1, None) == lb.ERR_ARG
    assert lib.lbdd_road_cm(4, None, a16, a16, 1, a16, 1, a16, a16, 1, None) == lb.ERR_ARG


def test_max_centers(lb):
    """The k limit is host arithmetic over the solver's shared-memory layout:
    below the 227 KB a CTA may use, whatever the stored CM width."""
    k = lb.max_centers()
    assert k == 5376


def test_tune_table_arguments(lb, lib):
    d = ctypes.c_double()
    for C in (0, 3, 32):
        assert lib.lbdd_tune_get(lb.CM_I32, 100, C, ctypes.byref(d)) == lb.ERR_ARG
    assert lib.lbdd_tune_get(lb.CM_I32, 0, 1, ctypes.byref(d)) == lb.ERR_ARG
    assert lib.lbdd_tune_get(lb.CM_I32, 100, 1, None) == lb.ERR_ARG
    assert lib.lbdd_tune_clear() == lb.OK


@no_gpu
def test_valid_calls_fail_without_a_gpu(lb, lib):
    inst = L.make_named("tiny")
    h = ctypes.c_void_p()
    cm = np.ascontiguousarray(inst.cm)
    rc = lib.lbdd_create(ctypes.byref(h), inst.n, inst.k, _ptr(cm), lb.CM_I32, 0,
                         _ptr(inst.cap), _ptr(inst.pen), None)
    assert rc in (lb.ERR_CUDA, lb.ERR_NODEV) and h.value is None
    if rc == lb.ERR_CUDA:
        assert lib.lbdd_last_cuda_error()         # names the failing runtime call
    cfg = lb._ServerConfig(1 << 30, 0, 0, 0)
    s = ctypes.c_void_p()
    assert lib.lbdd_server_create(ctypes.byref(s), ctypes.byref(cfg)) in (lb.ERR_CUDA,
                                                                         lb.ERR_NODEV)
    assert s.value is None


@no_gpu
def test_binding_raises_without_a_gpu(lb):
    """The product path has no CPU fallback: every entry point raises."""
    inst = L.make_named("tiny")
    with pytest.raises(lb.LbddError):
        lb.Solver(inst.cm, inst.cap, inst.pen)
    with pytest.raises(lb.LbddError):
        lb.Solver(inst.cm, inst.cap, None, strict=True)
    with pytest.raises(lb.LbddError):
        lb.Server(1 << 30)
    with pytest.raises(lb.LbddError):
        lb.tune_get(lb.CM_I32, 20, 1)


def test_binding_checks_buffer_sizes(lb):
    """The C side reads exactly n*k costs and k capacities and penalties: the
    binding refuses arrays of other sizes before calling it."""
    cm = np.ones((4, 3), np.int32)
    ones3 = np.ones(3, np.int32)
    with pytest.raises(ValueError):
        lb.create(4, 3, cm, ones3[:2], ones3)
    with pytest.raises(ValueError):
        lb.create(4, 3, cm, ones3, np.ones(4, np.int32))
    with pytest.raises(ValueError):
        lb.create(5, 3, cm, ones3, ones3)
    with pytest.raises(ValueError):
        lb.create_strict(5, 3, cm, ones3)
    with pytest.raises(ValueError):
        lb.set_penalty_table(None, np.ones((3, 2), np.int32), k=4)
    with pytest.raises(ValueError):
        lb.set_penalty_table(None, np.ones(3, np.int32))
