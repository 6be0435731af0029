"""The allocation-free best-transfer entry point (lbdd_best_transfer_noalloc).

Callers that may not allocate device memory get the table from a fixed
device array instead of a workspace.  This file is collected last on purpose,
so that a run stopping at the first failure has already run everything else.
The test passes both alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import lbdd_inputs as L
import oracle

pytestmark = pytest.mark.gpu


def _noalloc_fn(lib):
    f = lib.lbdd_best_transfer_noalloc
    P = ctypes.c_void_p
    f.argtypes = [ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int, ctypes.c_int64, P, P, P, P]
    f.restype = ctypes.c_int
    return f


def _device_cm(lb, inst, cm_dtype):
    import torch
    np_dt, t_dt = (np.int16, torch.int16) if cm_dtype == lb.CM_I16 else (np.int32, torch.int32)
    ld = lb.cm_pitch(inst.k, cm_dtype)
    buf = torch.zeros(inst.n * ld + 128, dtype=t_dt, device="cuda")
    host = np.zeros((inst.n, ld), np_dt)
    host[:, :inst.k] = inst.cm.astype(np_dt)
    buf[: inst.n * ld].copy_(torch.from_numpy(host.reshape(-1)))
    return buf, ld


def test_noalloc_matches_workspace_entry_point_twice(gpu_lib):
    import torch
    lib = gpu_lib.load()
    noalloc = _noalloc_fn(lib)
    # calls in a row on different instances: each must not see anything the
    # one before it left in the shared scratch; the last has int32 costs
    # (the int32 scan reads up to 128 entries past the last row)
    cases = [(L.random_small(9100, n=30000, k=130, cm_max=400), gpu_lib.CM_I16),
             (L.random_small(9101, n=7000, k=37, cm_max=9), gpu_lib.CM_I16),
             (L.random_small(9102, n=5000, k=61, cm_max=100000), gpu_lib.CM_I32)]
    for inst, cm_dtype in cases:
        buf, ld = _device_cm(gpu_lib, inst, cm_dtype)
        smin, _ = oracle.smin_order(inst.cm)
        assign = smin.copy()
        assign[::5] = -1
        a = torch.from_numpy(assign).cuda()
        k = inst.k
        tc_ref = torch.empty(k * k, dtype=torch.int32, device="cuda")
        td_ref = torch.empty_like(tc_ref)
        wsb = gpu_lib.best_transfer_workspace(inst.n, k)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        gpu_lib.best_transfer(inst.n, k, buf, cm_dtype, ld, a, tc_ref, td_ref, ws, wsb)
        tc = torch.full((k * k,), 7, dtype=torch.int32, device="cuda")
        td = torch.full((k * k,), 7, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        rc = noalloc(inst.n, k, buf.data_ptr(), cm_dtype, ld, a.data_ptr(), tc.data_ptr(),
                     td.data_ptr(), stream)
        assert rc == 0, gpu_lib.strerror(rc)
        torch.cuda.synchronize()
        assert torch.equal(tc, tc_ref) and torch.equal(td, td_ref)
        # and both equal the oracle's table for the same allotment
        rtc, rtd = oracle.best_transfer(inst.cm, assign)
        rtc = np.where(rtc >= oracle.INF, 2**31 - 1, rtc)
        assert np.array_equal(tc.cpu().numpy().reshape(k, k), rtc)
        assert np.array_equal(td.cpu().numpy().reshape(k, k), rtd)


def test_noalloc_rejects_oversized_request(gpu_lib):
    lib = gpu_lib.load()
    noalloc = _noalloc_fn(lib)
    n, k = 10_000_000, 2000         # needs more than the fixed 64 MiB
    assert gpu_lib.best_transfer_workspace(n, k) > (64 << 20)
    rc = noalloc(n, k, 16, gpu_lib.CM_I16, 2000, 16, 16, 16, None)
    assert rc == gpu_lib.ERR_BUDGET
