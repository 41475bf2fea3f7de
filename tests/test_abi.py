"""The C-ABI library loads, exports every symbol include/fk.h declares, and
rejects invalid arguments on the host before any CUDA call (no GPU needed:
none of these calls launches work)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2104_14561_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2104_14561_gb300.build import build
        build()
    _lib.load()
    return _lib


def _declared():
    txt = open(os.path.join(ROOT, "include", "fk.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fk_[a-z_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(L):
    lib = L.load()
    names = _declared()
    assert set(names) == set(L.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


_KEEP = []


def _args(L, **kw):
    g = L.Grid()
    g.dim = kw.get("dim", 2)
    n = kw.get("n", (33, 17))
    for m in range(len(n)):
        g.n[m] = n[m]
        g.lo[m] = kw.get("lo", (0.0, 0.0, 0.0))[m]
        g.hi[m] = kw.get("hi", (2.0, 1.0, 1.0))[m]
    for m, ax in enumerate(kw.get("axes", ())):
        if ax is not None:
            arr = (ctypes.c_double * len(ax))(*ax)
            _KEEP.append(arr)
            g.axis[m] = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
    r = L.Region(kw.get("faces", L.FK_ALL_FACES_ABSORBING))
    c = L.Coeffs()
    c.family = kw.get("family", L.FK_CELLULAR_FLOW)
    for k, v in enumerate(kw.get("p", (1.0, 0.2, 2 * math.pi, 1e-3))):
        c.p[k] = v
    return g, r, c


RUNAWAY = (0.3, 1e5, 1.0, 0.042, 1.0, 1.0, 0.7, 1e-2, 20.0, 0.003, 1e-4)

CASES = [
    (dict(dim=0), 1),
    (dict(dim=4), 1),
    (dict(n=(2, 17)), 1),
    (dict(dt=0.0), 1),
    (dict(dt=-1e-3), 1),
    (dict(dt=float("nan")), 1),
    (dict(n_steps=0), 1),
    (dict(prec=7), 1),
    (dict(path=9), 1),
    (dict(family=5), 1),
    (dict(p=(1.0, float("inf"), 1.0, 1e-3)), 1),
    (dict(p=(1.0, 0.2, 1.0, -1e-3)), 1),
    (dict(q=0), 2),
    (dict(q=9), 2),
    (dict(faces=0x3), 2),
    (dict(path=1), 2),             # CSR with a time-dependent drift
    (dict(dim=3, n=(5, 5, 5)), 1),  # the cellular flow is two-dimensional
    # d = 3: constant drift, uniform, absorbing, matrix-free, narrow point spread
    (dict(dim=3, n=(9, 9, 9), family=0, p=(0.1, 0, 0, 1.0), faces=0x3C), 2),
    (dict(dim=3, n=(9, 9, 9), family=0, p=(0.1, 0, 0, 1.0), path=1), 2),
    (dict(dim=3, n=(5, 5, 5), family=0, p=(0.1, 0, 0, 1.0),
          axes=(None, None, [0.0, 0.1, 0.5, 0.7, 1.1])), 1),  # last coordinate != hi
    (dict(dim=3, n=(9, 9, 9), family=0, p=(0.1, 0, 0, 1.0), dt=0.05), 2),  # span > 6 cells
    (dict(dim=3, n=(4, 33, 33), family=0, p=(0.1, 0, 0, 0.3), dt=2e-3), 2),  # n < W on x
    # the runaway model: d = 3, p > 0, xi within [-1, 1], positive scales
    (dict(family=3, p=RUNAWAY), 1),  # two-dimensional grid
    (dict(dim=3, n=(9, 9, 9), family=3, p=RUNAWAY, lo=(0.0, -1.0, 0.0), hi=(50, 1, 1)), 1),
    (dict(dim=3, n=(9, 9, 9), family=3, p=RUNAWAY, lo=(2.0, -1.5, 0.0), hi=(50, 1, 1)), 1),
    (dict(dim=3, n=(9, 9, 9), family=3, p=RUNAWAY[:1] + (0.0,) + RUNAWAY[2:],
          lo=(2.0, -1.0, 0.0), hi=(50, 1, 1)), 1),  # tau = 0
    (dict(dim=3, n=(9, 9, 9), family=3, p=RUNAWAY, lo=(2.0, -1.0, 0.0), hi=(50, 1, 1),
          path=1), 2),
    (dict(dim=3, n=(9, 65, 9), family=3, p=RUNAWAY, lo=(2.0, -1.0, 0.0), hi=(50, 1, 1),
          dt=0.5), 2),  # the xi points span more than 6 cells
    (dict(dim=1, n=(33,)), 1),     # the cellular flow is two-dimensional
    (dict(family=2, dim=1, n=(33,), p=(10.0, 2.0, 0.15, 0.6)), 1),  # so is the paper's
    (dict(faces=0x3C, dim=1, n=(33,), family=0, p=(0.1, 0, 0, 1.0)), 2),  # periodic x in 1D
    (dict(faces=0x3C, path=1, p=(1.0, 0.0, 1.0, 1e-3)), 2),  # periodic x on the CSR path
    (dict(faces=0x33), 2),         # periodic y is not offered
    (dict(family=2, path=1, p=(10.0, 2.0, 0.0, 0.6)), 2),  # the paper's flow: matrix-free only
    # non-uniform axes
    (dict(n=(5, 3), axes=([0.0, 0.5, 1.0, 1.5, 2.1], None)), 1),  # last coordinate != hi
    (dict(n=(5, 3), axes=([0.0, 0.5, 0.5, 1.5, 2.0], None)), 1),  # not increasing
    (dict(n=(5, 3), axes=([0.0, 0.2, 1.0, 1.5, 2.0], None), faces=0x3C), 2),  # with periodic x
    (dict(n=(5, 3), axes=([0.0, 0.2, 1.0, 1.5, 2.0], None), path=1,
          p=(1.0, 0.0, 1.0, 1e-3)), 2),  # on the CSR path
    (dict(dim=1, n=(5,), axes=([0.0, 0.2, 1.0, 1.5, 2.1],), family=0, p=(0.1, 0, 0, 1.0)), 1),
]


@pytest.mark.parametrize("kw,status", CASES)
def test_plan_create_rejects(L, kw, status):
    lib = L.load()
    g, r, c = _args(L, **kw)
    h = ctypes.c_void_p()
    st = lib.fk_plan_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(r), ctypes.byref(c),
                            kw.get("q", 6), kw.get("dt", 1e-3), kw.get("n_steps", 10),
                            kw.get("prec", 0), kw.get("path", 0))
    assert st == status
    assert h.value is None


def test_null_arguments(L):
    lib = L.load()
    g, r, c = _args(L)
    assert lib.fk_plan_create(None, ctypes.byref(g), ctypes.byref(r), ctypes.byref(c), 6, 1e-3,
                              10, 0, 0) == 1
    h = ctypes.c_void_p()
    assert lib.fk_plan_create(ctypes.byref(h), None, ctypes.byref(r), ctypes.byref(c), 6, 1e-3,
                              10, 0, 0) == 1
    assert lib.fk_solve(None, None, None, None, 0, None) == 1
    assert lib.fk_march(None, 1, 0, None, None, None) == 1
    assert lib.fk_plan_get_info(None, None) == 1
    assert lib.fk_last_device_error(None) == 1
    assert lib.fk_plan_destroy(None) == 0
    a = (ctypes.c_double * 4)()
    assert lib.fk_gauss_hermite(0, a, a) == 1
    assert lib.fk_gauss_hermite(17, a, a) == 1
    assert lib.fk_gauss_hermite(4, None, a) == 1


def test_status_strings(L):
    lib = L.load()
    for code, name in L.STATUS.items():
        assert lib.fk_status_string(code).decode().startswith(name)
    assert b"unknown" in lib.fk_status_string(99)


def test_static_entry_rejects_axes(L):
    """fk_solve_static marches uniform meshes only; coordinates are refused
    on the host, before any CUDA call."""
    lib = L.load()
    lib.fk_solve_static.argtypes = [ctypes.POINTER(L.Grid), ctypes.POINTER(L.Coeffs), ctypes.c_int,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]
    lib.fk_solve_static.restype = ctypes.c_int
    g, _, c = _args(L, n=(5, 3), axes=([0.0, 0.2, 1.0, 1.5, 2.0], None))
    st = lib.fk_solve_static(ctypes.byref(g), ctypes.byref(c), 4, 1e-3, 5, 0, None,
                             ctypes.c_void_p(256), None)
    assert st == 2


QUENCH = (0.1, 6000.0, 1.0, 3.0, 0.005, 3.0, 0.5, 0.0, 1e-4, 2.0, 0.0, 0.01, 511.0)


def test_runaway_quench_params_match_oracle(L, oracle):
    """The library's thermal-quench schedule (host code, no GPU) against the
    oracle's, written separately: the same constants at every time."""
    lib = L.load()
    q = (ctypes.c_double * 16)(*QUENCH)
    out = (ctypes.c_double * 11)()
    for t in (0.0, 0.05, 0.7, 3.0, 40.0):
        assert lib.fk_runaway_quench_params(q, t, out) == 0
        np.testing.assert_allclose(list(out), oracle.quench_params(QUENCH, t), rtol=1e-15,
                                   atol=0.0)
    assert lib.fk_runaway_quench_params(None, 0.0, out) == 1
    assert lib.fk_runaway_quench_params(q, float("nan"), out) == 1
    bad = (ctypes.c_double * 16)(*QUENCH)
    bad[6] = 0.0  # t_star
    assert lib.fk_runaway_quench_params(bad, 0.0, out) == 1


@pytest.mark.parametrize("kw,status", [
    (dict(family=4, p=QUENCH), 1),  # two-dimensional grid
    (dict(dim=3, n=(9, 9, 9), family=4, p=QUENCH[:3] + (0.0,) + QUENCH[4:],
          lo=(2.0, -1.0, 0.0), hi=(8.0, 1.0, 1.0)), 1),  # T0 = 0
    (dict(dim=3, n=(9, 9, 9), family=4, p=QUENCH[:12] + (-511.0,),
          lo=(2.0, -1.0, 0.0), hi=(8.0, 1.0, 1.0)), 1),  # mc2 < 0
    (dict(dim=3, n=(9, 9, 9), family=4, p=QUENCH[:4] + (1e-8,) + QUENCH[5:],
          lo=(2.0, -1.0, 0.0), hi=(8.0, 1.0, 1.0)), 1),  # ln Lambda(Tf) < 0
    (dict(dim=3, n=(9, 9, 9), family=4, p=QUENCH, lo=(2.0, -1.0, 0.0), hi=(8.0, 1.0, 1.0),
          path=1), 2),
])
def test_plan_create_rejects_quench(L, kw, status):
    test_plan_create_rejects(L, kw, status)
