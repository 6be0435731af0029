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


def _check_sampled_rows(inst, assign, tc, td, centers):
    for u in centers:
        members = np.nonzero(assign == u)[0]
        if len(members) == 0:
            assert (tc[u] == 2**31 - 1).all() and (td[u] == -1).all()
            continue
        rows = inst.cm[members].astype(np.int64)
        t = rows - rows[:, [u]]
        best = t.argmin(axis=0)               # first minimum: lowest d on equal cost
        exp_t = t[best, np.arange(inst.k)]
        exp_d = members[best]
        exp_t[u], exp_d[u] = 2**31 - 1, -1
        assert np.array_equal(tc[u], exp_t) and np.array_equal(td[u], exp_d)


def _check_witnesses(inst, assign, tc, td):
    """Every finite entry names a unit of its row's center whose transfer
    costs exactly that much; every empty center's row is empty."""
    k = inst.k
    u, v = np.nonzero(td >= 0)
    d = td[u, v]
    assert (assign[d] == u).all() and (u != v).all()
    cost = inst.cm[d, v].astype(np.int64) - inst.cm[d, u].astype(np.int64)
    assert np.array_equal(cost, tc[u, v].astype(np.int64))
    empty = np.bincount(assign[assign >= 0], minlength=k) == 0
    assert (td[empty] == -1).all() and (tc[empty] == 2**31 - 1).all()
    assert (np.diag(td) == -1).all()


def test_large_snapshot_full_size(gpu_lib):
    """The 2,000,000 x 2,000 instance at the size the scan benchmark times,
    every unit at its s_min, int16 and int32 storage: the two tables are
    equal, every entry's witness is consistent, and sampled rows equal the
    definition (a plain loop over that center's units)."""
    import torch
    lb = gpu_lib
    inst = L.make_named("large", dtype="i16")
    n, k = inst.n, inst.k
    smin = inst.cm.argmin(axis=1).astype(np.int32)    # first minimum: lowest center index
    ld16, ld32 = lb.cm_pitch(k, lb.CM_I16), lb.cm_pitch(k, lb.CM_I32)
    assert ld16 == k and ld32 == k                     # unpadded rows: one host copy serves both
    cm16 = torch.zeros(n * k + 128, dtype=torch.int16, device="cuda")
    cm16[: n * k].copy_(torch.from_numpy(inst.cm.reshape(-1)))
    a = torch.from_numpy(smin).cuda()
    wsb = lb.best_transfer_workspace(n, k)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")

    def table(buf, cmd):
        tc = torch.empty(k * k, dtype=torch.int32, device="cuda")
        td = torch.empty(k * k, dtype=torch.int32, device="cuda")
        lb.best_transfer(n, k, buf, cmd, k, a, tc, td, ws, wsb)
        torch.cuda.synchronize()
        return tc.cpu().numpy().reshape(k, k), td.cpu().numpy().reshape(k, k)

    tc, td = table(cm16, lb.CM_I16)
    cm32 = cm16.to(torch.int32)
    del cm16
    tc32, td32 = table(cm32, lb.CM_I32)
    del cm32
    assert np.array_equal(tc, tc32) and np.array_equal(td, td32)
    _check_witnesses(inst, smin, tc, td)
    rng = np.random.default_rng(3)
    _check_sampled_rows(inst, smin, tc, td, rng.choice(k, 16, replace=False))


# Row widths on both sides of the 512-byte switch between the register scan
# and the bulk-copy scan, both ends of the row-order path (256 to 512 centers,
# int16 and int32, several row ranges), the largest k of each storage type, and allotments
# with many equal costs (scale 3: CM in 1..6) where one center holds most
# units, so that its rows are split over many work items and equal-cost
# candidates from different items meet in the table merge.
SHAPE_CASES = [  # (n, k, dtype, scale, skew)
    (9000, 256, "i16", 100.0, False),     # 512-byte rows: bulk copies
    (9000, 248, "i16", 100.0, False),     # 496-byte rows: register scan
    (9000, 128, "i32", 100.0, False),
    (9000, 124, "i32", 100.0, False),
    (6000, 4096, "i16", 1000.0, False),   # largest int16 k: one row group
    (6000, 2048, "i32", 1000.0, False),   # largest int32 k
    (40000, 300, "i16", 3.0, True),
    (40000, 300, "i32", 3.0, True),
    (40000, 40, "i16", 3.0, True),
    (2, 600, "i16", 3.0, False),
    (140000, 512, "i16", 3.0, True),      # row-order path: three row ranges at least, ties
    (3, 300, "i16", 100.0, False),        # row-order path with one row per range
    (70000, 513, "i16", 100.0, True),     # just past the row-order path: row gathers
    (140000, 512, "i32", 3.0, True),      # int32 row-order path (64-bit keys), ties
    (3, 300, "i32", 100.0, False),        # int32 row-order path, one range
    (1, 300, "i32", 100.0, False),        # one unit: no int32 range fits, row gathers
]


@pytest.mark.parametrize("case", range(len(SHAPE_CASES)))
def test_scan_shapes_and_ties(gpu_lib, case):
    n, k, dtype, scale, skew = SHAPE_CASES[case]
    inst = L.make_named("city", dtype=dtype, n=n, k=k, seed=8100 + case, scale=scale,
                        cap_frac=max(0.8, 2.0 * k / n))   # capacities need a total >= k
    assert inst.cm.min() >= 1
    assign = inst.cm.argmin(axis=1).astype(np.int32)
    if skew:
        rng = np.random.default_rng(case)
        assign[rng.random(n) < 0.6] = 3 % k        # one center takes ~60% of the units
        assign[rng.random(n) < 0.05] = -1
    tc, td = gpu_table(gpu_lib, inst, assign, dtype)
    rtc, rtd = ref_table(inst, assign)
    assert np.array_equal(tc, rtc)
    assert np.array_equal(td, rtd)
    assert (td != -2).all()                        # no scan wait ran out


def test_scan_repeated_calls_share_a_workspace(gpu_lib):
    """Two different allotments through one workspace, int16 then int32: each
    call rewrites every scratch word it reads."""
    import torch
    lb = gpu_lib
    inst = L.make_named("city", dtype="i16", n=20000, k=500, seed=8200, scale=50.0)
    n, k = inst.n, inst.k
    wsb = lb.best_transfer_workspace(n, k)
    ws = torch.full((wsb,), 0x5A, dtype=torch.uint8, device="cuda")
    a1 = inst.cm.argmin(axis=1).astype(np.int32)
    a2 = np.random.default_rng(1).integers(-1, k, n).astype(np.int32)
    for dtype, assign in (("i16", a1), ("i32", a2), ("i16", a2), ("i32", a1)):
        cmd = lb.CM_I16 if dtype == "i16" else lb.CM_I32
        tdt = torch.int16 if dtype == "i16" else torch.int32
        ld = lb.cm_pitch(k, cmd)
        host = np.zeros((n, ld), inst.cm.dtype if dtype == "i16" else np.int32)
        host[:, :k] = inst.cm
        buf = torch.zeros(n * ld + 128, dtype=tdt, device="cuda")
        buf[: n * ld].copy_(torch.from_numpy(host.reshape(-1)).to(tdt))
        a = torch.from_numpy(assign).cuda()
        tc = torch.empty(k * k, dtype=torch.int32, device="cuda")
        td = torch.empty(k * k, dtype=torch.int32, device="cuda")
        lb.best_transfer(n, k, buf, cmd, ld, a, tc, td, ws, wsb)
        torch.cuda.synchronize()
        rtc, rtd = ref_table(inst, assign)
        assert np.array_equal(tc.cpu().numpy().reshape(k, k), rtc)
        assert np.array_equal(td.cpu().numpy().reshape(k, k), rtd)
