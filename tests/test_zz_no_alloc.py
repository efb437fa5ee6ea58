"""dg_max_dt_noalloc: the CFL time step for callers that cannot allocate
device memory (inside CUDA graph capture, or under an application memory
manager that owns the device), checked through the C ABI against the
handle-based dg_max_dt and the FP64 oracle on the same state, on two calls in
a row, with the device's free memory unchanged across those calls.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test before this one.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2303_11767_gb300 import dgswe, synth

pytestmark = pytest.mark.gpu

CFL = 0.1


@pytest.mark.parametrize("nlon,nlat,p,seed", [(20, 10, 1, 1), (36, 18, 3, 6), (15, 19, 4, 2)])
def test_max_dt_noalloc_matches_dg_max_dt(nlon, nlat, p, seed):
    torch = pytest.importorskip("torch")
    L = dgswe.lib()
    o = O.Oracle.sphere(nlon, nlat, p, dgswe.EARTH_RADIUS, dgswe.GRAVITY, dgswe.OMEGA)
    u = o.project_tensor(synth.SmoothField(seed).fields_grid)
    want_oracle = o.max_dt(u, CFL)
    with dgswe.Solver(nlon, nlat, p, precision="fp64") as s:
        s.set_state(u)
        want = s.max_dt(CFL)
    d_u = torch.tensor(np.ascontiguousarray(u).reshape(-1), dtype=torch.float64, device="cuda")
    d_dt = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        st = L.dg_max_dt_noalloc(ctypes.c_void_p(d_u.data_ptr()), nlon, nlat, p, dgswe.EARTH_RADIUS,
                                 dgswe.GRAVITY, CFL, ctypes.c_void_p(d_dt.data_ptr()), stream)
        assert st == dgswe.DG_OK, L.dg_last_error(None)

    d_dt.fill_(float("nan"))               # warm-up: loads every kernel used below once
    call()                                  # the first call on the device does the set-up
    torch.cuda.synchronize()
    assert abs(d_dt.item() / want - 1) < 1e-12
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(2):                      # two calls in a row share the scratch array
        d_dt.fill_(float("nan"))
        call()
        torch.cuda.synchronize()
        got = d_dt.item()
        assert abs(got / want - 1) < 1e-12, (got, want)
        assert abs(got / want_oracle - 1) < 1e-12, (got, want_oracle)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0, (free0, free1)


def test_max_dt_noalloc_rejects_oversize_and_reports_bad_depth():
    torch = pytest.importorskip("torch")
    L = dgswe.lib()
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    big = 8192 + 1                          # one row more than the scratch holds
    st = L.dg_max_dt_noalloc(ctypes.c_void_p(d.data_ptr()), 4, big, 1, 1.0, 1.0, CFL,
                             ctypes.c_void_p(d.data_ptr()), None)
    assert st == dgswe.DG_EINVAL
    assert b"scratch limit" in L.dg_last_error(None)
    # negative depth everywhere -> -1
    nlon, nlat, p = 8, 4, 1
    u = np.zeros((nlat, nlon, 3, 4))
    u[..., 0, 0] = -2.0
    d_u = torch.tensor(u.reshape(-1), dtype=torch.float64, device="cuda")
    d_dt = torch.empty(1, dtype=torch.float64, device="cuda")
    st = L.dg_max_dt_noalloc(ctypes.c_void_p(d_u.data_ptr()), nlon, nlat, p, 1.0, 1.0, CFL,
                             ctypes.c_void_p(d_dt.data_ptr()), None)
    assert st == dgswe.DG_OK
    torch.cuda.synchronize()
    assert d_dt.item() == -1.0
    # a NaN in one momentum mode of one element (h stays positive) -> -1
    u = np.zeros((nlat, nlon, 3, 4))
    u[..., 0, 0] = 2.0
    u[2, 5, 1, 3] = float("nan")
    d_u = torch.tensor(u.reshape(-1), dtype=torch.float64, device="cuda")
    d_dt.fill_(0.0)
    st = L.dg_max_dt_noalloc(ctypes.c_void_p(d_u.data_ptr()), nlon, nlat, p, 1.0, 1.0, CFL,
                             ctypes.c_void_p(d_dt.data_ptr()), None)
    assert st == dgswe.DG_OK
    torch.cuda.synchronize()
    assert d_dt.item() == -1.0
