"""GPU tests of the request server (continuous batching).

Each request's allotment and objective must be the oracle's and the same as
the instance solved alone on the GPU, however its rounds were sliced into
passes and whatever else shared those passes.
"""
import numpy as np
import pytest

import lbdd_inputs as L
import oracle

pytestmark = pytest.mark.gpu

TIMEOUT_MS = 300_000


def requests(count, seed0=500):
    return [L.make(L.batch_recipe(seed0 + i, n_range=(2.3, 3.4), k_range=(0.4, 2.2)),
                   dtype="i16" if i % 2 else "i32") for i in range(count)]


@pytest.fixture(scope="module")
def reqs():
    insts = requests(24)
    refs = [oracle.asral(x.cm, x.cap, x.pen) for x in insts]
    return insts, refs


def test_served_equals_alone_and_oracle(gpu_lib, reqs):
    insts, refs = reqs
    alone = []
    for x in insts[:6]:
        with gpu_lib.Solver(x.cm, x.cap, x.pen) as s:
            s.solve()
            alone.append((s.assignment(), s.objective))
    # a short quantum: most requests span several passes
    with gpu_lib.Server(budget_bytes=8 << 30, max_active=12, quantum_us=300) as srv:
        tickets = [srv.submit(x.cm, x.cap, x.pen) for x in insts]
        for i, t in enumerate(tickets):
            info, a = srv.result(t, TIMEOUT_MS)
            assert info.state == gpu_lib.REQ_DONE and info.status == 0
            assert info.objective == refs[i].delta
            assert np.array_equal(a, refs[i].assign)
            assert info.submit_ns <= info.admit_ns <= info.done_ns
            if i < len(alone):
                assert np.array_equal(a, alone[i][0]) and info.objective == alone[i][1]
        st = srv.stats()
        assert st.completed == len(insts) and st.failed == 0
        assert st.passes > 1 and st.peak_active <= 12
        assert st.bytes_in_use == 0


def test_budget_serialises_admission(gpu_lib, reqs):
    """A budget that holds one request at a time still serves all of them."""
    insts, refs = reqs
    sub = insts[:5]
    one = max(x.n * x.k * 4 for x in sub) * 2 + (64 << 20)
    with gpu_lib.Server(budget_bytes=one, quantum_us=2000) as srv:
        tickets = [srv.submit(x.cm, x.cap, x.pen) for x in sub]
        for i, t in enumerate(tickets):
            info, a = srv.result(t, TIMEOUT_MS)
            assert info.state == gpu_lib.REQ_DONE
            assert info.objective == refs[i].delta and np.array_equal(a, refs[i].assign)
        st = srv.stats()
        assert st.peak_bytes <= one


def test_request_over_budget_fails_cleanly(gpu_lib):
    x = L.random_small(9, n=2000, k=40)
    with gpu_lib.Server(budget_bytes=1 << 16) as srv:    # below one request's footprint
        t = srv.submit(x.cm, x.cap, x.pen)
        info, _ = srv.result(t, TIMEOUT_MS)
        assert info.state == gpu_lib.REQ_FAILED and info.status == gpu_lib.ERR_BUDGET


def test_submit_refuses_too_many_centers(gpu_lib):
    k = gpu_lib.max_centers() + 1
    cm = np.ones((2, k), np.int32)
    ones = np.ones(k, np.int32)
    with gpu_lib.Server(budget_bytes=1 << 30) as srv:
        with pytest.raises(gpu_lib.LbddError) as e:
            srv.submit(cm, ones, ones)
        assert e.value.code == gpu_lib.ERR_ARG
        assert srv.stats().queued == 0


def test_destroy_with_work_outstanding(gpu_lib, reqs):
    insts, _ = reqs
    srv = gpu_lib.Server(budget_bytes=8 << 30, max_active=4, quantum_us=500)
    for x in insts:
        srv.submit(x.cm, x.cap, x.pen)
    srv.close()                       # returns: queued requests dropped, pass ends at its quantum


def test_device_resident_requests_and_aging(gpu_lib, reqs):
    """Requests whose CM is already in device memory (lbdd_server_submit_ex)
    give the oracle's results.  Then a long request shares one cluster-size
    group (16 CTAs forced) with twelve short ones under a 100 us quantum, so
    shortest-first ordering and aging both reorder the group between passes;
    every result is still the oracle's."""
    import torch
    insts, refs = reqs
    with gpu_lib.Server(budget_bytes=8 << 30, max_active=12, quantum_us=300) as srv:
        tickets = [srv.submit(torch.from_numpy(x.cm).cuda(), x.cap, x.pen) for x in insts[:8]]
        for i, t in enumerate(tickets):
            info, a = srv.result(t, TIMEOUT_MS)
            assert info.state == gpu_lib.REQ_DONE and info.status == 0
            assert info.objective == refs[i].delta and np.array_equal(a, refs[i].assign)
    big = L.make(L.Recipe(n=6000, k=300, seed=4242, cap_frac=0.8, pen=(50, 500), name="big"),
                 dtype="i16")
    small = [L.make(L.Recipe(n=600, k=300, seed=4300 + i, cap_frac=0.8, pen=(50, 500),
                             name=f"s{i}"), dtype="i16") for i in range(12)]
    ref_big = oracle.asral(big.cm, big.cap, big.pen)
    refs_small = [oracle.asral(x.cm, x.cap, x.pen) for x in small]
    with gpu_lib.Server(budget_bytes=8 << 30, quantum_us=100, cluster_size=16) as srv:
        tb = srv.submit(big.cm, big.cap, big.pen)
        ts = [srv.submit(x.cm, x.cap, x.pen) for x in small]
        info, a = srv.result(tb, TIMEOUT_MS)
        assert info.objective == ref_big.delta and np.array_equal(a, ref_big.assign)
        for t, r in zip(ts, refs_small):
            info, a = srv.result(t, TIMEOUT_MS)
            assert info.objective == r.delta and np.array_equal(a, r.assign)


def test_submit_ex_rejects_bad_location_flag(gpu_lib):
    import ctypes
    x = L.random_small(10, n=50, k=4)
    lib = gpu_lib.load()
    out = np.empty(50, np.int32)
    t = ctypes.c_int64()
    cap, pen = x.cap.astype(np.int32), x.pen.astype(np.int32)
    with gpu_lib.Server(budget_bytes=1 << 30) as srv:
        rc = lib.lbdd_server_submit_ex(srv.h, 50, 4, x.cm.ctypes.data, gpu_lib.CM_I32, 2,
                                       cap.ctypes.data, pen.ctypes.data, out.ctypes.data,
                                       ctypes.byref(t))
        assert rc == gpu_lib.ERR_ARG
