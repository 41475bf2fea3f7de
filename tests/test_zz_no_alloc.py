"""fk_solve_static: the march for callers that cannot allocate device memory.

Such callers (a host application whose pool allocator owns all device
memory, latency-bound loops that cannot absorb cudaMalloc's
synchronisation) get an entry point whose scratch lives in a static device
array instead of plan memory.  Its results must equal fk_solve's within the
parity tolerances (1e-5 FP32, 1e-12 FP64), on two calls in a row (the second
call reuses the array the first one left behind); its error word, read back
with fk_static_last_device_error, must be clear; and a call after the
one-time set-up must leave the device's free memory unchanged.  This file is
collected last so that a failure here does not hide the other tests.
"""
import ctypes
import math

import pytest

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_14561_gb300 import _lib as L
    from paper_2104_14561_gb300 import fk
    lib = L.load()
    lib.fk_solve_static.argtypes = [ctypes.POINTER(L.Grid), ctypes.POINTER(L.Coeffs), ctypes.c_int,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]
    lib.fk_solve_static.restype = ctypes.c_int
    lib.fk_static_last_device_error.argtypes = []
    lib.fk_static_last_device_error.restype = ctypes.c_int
    return torch, L, fk, lib


def _structs(L, n, params):
    g = L.Grid()
    g.dim = 2
    g.n[0], g.n[1] = n
    g.lo[0], g.lo[1] = 0.0, 0.0
    g.hi[0], g.hi[1] = 2.0, 1.0
    c = L.Coeffs()
    c.family = L.FK_CELLULAR_FLOW
    for k, v in enumerate(params):
        c.p[k] = v
    return g, c


@pytest.mark.parametrize("precision,n_steps", [("fp32", 2000), ("fp64", 200)])
def test_static_scratch_matches_fk_solve(env, precision, n_steps):
    torch, L, fk, lib = env
    n, q, dt = (1025, 513), 6, 1e-3
    params = (1.0, 0.2, 2 * math.pi, 1e-3)
    plan = fk.Plan(fk.PlanSpec(n=n, lo=(0.0, 0.0), hi=(2.0, 1.0), family="cellular_flow",
                               params=params, q=q, dt=dt, n_steps=n_steps, precision=precision))
    ref = plan.solve()
    torch.cuda.synchronize()
    plan.close()
    g, c = _structs(L, n, params)
    prec = L.FK_FP32 if precision == "fp32" else L.FK_FP64
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full(ref.shape, float("nan"), dtype=ref.dtype, device="cuda")
        st = lib.fk_solve_static(ctypes.byref(g), ctypes.byref(c), q, dt, n_steps, prec, None,
                                 ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, L.STATUS.get(st, st)
        torch.cuda.synchronize()
        assert L.STATUS[lib.fk_static_last_device_error()] == "FK_OK"
        err = (out.double() - ref.double()).abs().max().item()
        assert err <= TOL[precision], (call, err)


def test_static_scratch_with_terminal_field_in_place(env):
    torch, L, fk, lib = env
    n, q, dt, n_steps = (257, 129), 5, 1e-3, 7
    params = (1.0, 0.2, 2 * math.pi, 1e-2)
    gen = torch.Generator().manual_seed(3)
    u0 = torch.rand((n[1], n[0]), generator=gen, dtype=torch.float64).cuda()
    plan = fk.Plan(fk.PlanSpec(n=n, lo=(0.0, 0.0), hi=(2.0, 1.0), family="cellular_flow",
                               params=params, q=q, dt=dt, n_steps=n_steps, precision="fp64"))
    ref = plan.solve(u0.clone())
    torch.cuda.synchronize()
    plan.close()
    g, c = _structs(L, n, params)
    for call in range(2):
        buf = u0.clone()
        st = lib.fk_solve_static(ctypes.byref(g), ctypes.byref(c), q, dt, n_steps, L.FK_FP64,
                                 ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        assert (buf - ref).abs().max().item() <= TOL["fp64"]


def test_static_scratch_rejects_oversize(env):
    torch, L, fk, lib = env
    out = torch.empty(1, device="cuda")
    g, c = _structs(L, (4097, 2049), (1.0, 0.2, 2 * math.pi, 1e-3))
    st = lib.fk_solve_static(ctypes.byref(g), ctypes.byref(c), 8, 5e-4, 10, L.FK_FP32, None,
                             ctypes.c_void_p(out.data_ptr()), None)
    assert L.STATUS[st] == "FK_ERR_INVALID_ARG"


def test_static_scratch_allocates_nothing(env):
    """After the first call on the device (the one-time set-up), a call must
    not change the device's free memory: every byte it uses is the static
    array or the caller's buffers."""
    torch, L, fk, lib = env
    n, q, dt, n_steps = (257, 129), 6, 1e-3, 20
    params = (1.0, 0.2, 2 * math.pi, 1e-3)
    g, c = _structs(L, n, params)
    out = torch.empty((n[1], n[0]), dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        st = lib.fk_solve_static(ctypes.byref(g), ctypes.byref(c), q, dt, n_steps, L.FK_FP32,
                                 None, ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, L.STATUS.get(st, st)
        torch.cuda.synchronize()

    call()  # set-up, if no earlier test made it
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        call()
    assert torch.cuda.mem_get_info()[0] == free0
    assert L.STATUS[lib.fk_static_last_device_error()] == "FK_OK"
