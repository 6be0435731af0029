"""GPU parity of the standalone best-transfer scan (lbdd_best_transfer).

Inputs are oracle-side only: the allotments are the oracle's s_min
assignment or the oracle's ASRAL result; expected tables are
oracle.best_transfer on the same allotment.
"""
import numpy as np
import pytest

import lbdd_inputs as L
import oracle

pytestmark = pytest.mark.gpu


def gpu_table(lb, inst, assign, dtype="i16"):
    import torch
    n, k = inst.n, inst.k
    cmd = lb.CM_I16 if dtype == "i16" else lb.CM_I32
    np_dt = np.int16 if dtype == "i16" else np.int32
    ld = lb.cm_pitch(k, cmd)
    buf = torch.zeros(n * ld + 128, dtype=torch.int16 if dtype == "i16" else torch.int32,
                      device="cuda")
    host = np.zeros((n, ld), np_dt)
    host[:, :k] = inst.cm.astype(np_dt)
    buf[: n * ld].copy_(torch.from_numpy(host.reshape(-1)))
    a = torch.from_numpy(np.ascontiguousarray(assign, np.int32)).cuda()
    tc = torch.empty(k * k, dtype=torch.int32, device="cuda")
    td = torch.empty(k * k, dtype=torch.int32, device="cuda")
    wsb = lb.best_transfer_workspace(n, k)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    lb.best_transfer(n, k, buf, cmd, ld, a, tc, td, ws, wsb)
    torch.cuda.synchronize()
    return tc.cpu().numpy().reshape(k, k), td.cpu().numpy().reshape(k, k)


def ref_table(inst, assign):
    tc, td = oracle.best_transfer(inst.cm, assign)
    return np.where(tc >= oracle.INF, 2**31 - 1, tc), td


@pytest.mark.parametrize("dtype", ["i16", "i32"])
@pytest.mark.parametrize("case", range(8))
def test_table_matches_oracle(gpu_lib, dtype, case):
    n = [1, 50, 4095, 4097, 9000, 20000, 70000, 3][case]
    k = [1, 7, 33, 64, 130, 257, 500, 2][case]
    inst = L.random_small(8000 + case, n=n, k=k, cm_max=[5, 60, 2000][case % 3])
    smin, _ = oracle.smin_order(inst.cm)
    assign = smin.copy()
    assign[::7] = -1                      # some units not allotted yet
    tc, td = gpu_table(gpu_lib, inst, assign, dtype)
    rtc, rtd = ref_table(inst, assign)
    assert np.array_equal(tc, rtc)
    assert np.array_equal(td, rtd)


def test_table_on_asral_allotment(gpu_lib):
    inst = L.make_named("tiny")
    res = oracle.asral(inst.cm, inst.cap, inst.pen)
    tc, td = gpu_table(gpu_lib, inst, res.assign)
    rtc, rtd = ref_table(inst, res.assign)
    assert np.array_equal(tc, rtc) and np.array_equal(td, rtd)


def test_city_snapshot_sampled_rows(gpu_lib):
    """City-scale CM (200,000 x 500) with every unit at its s_min: full GPU
    table; oracle rows for a sample of centers (each a plain loop over that
    center's units)."""
    inst = L.make_named("city", dtype="i16")
    smin, _ = oracle.smin_order(inst.cm)
    tc, td = gpu_table(gpu_lib, inst, smin)
    rng = np.random.default_rng(0)
    for u in rng.choice(inst.k, 12, replace=False):
        members = np.nonzero(smin == u)[0]
        if len(members) == 0:
            assert (tc[u] == 2**31 - 1).all() and (td[u] == -1).all()
            continue
        rows = inst.cm[members].astype(np.int64)
        t = rows - rows[:, [u]]
        # lexicographic (t, d): argmin returns the first (lowest d) minimum
        best = t.argmin(axis=0)
        exp_t = t[best, np.arange(inst.k)]
        exp_d = members[best]
        exp_t[u], exp_d[u] = 2**31 - 1, -1
        assert np.array_equal(tc[u], exp_t) and np.array_equal(td[u], exp_d)
