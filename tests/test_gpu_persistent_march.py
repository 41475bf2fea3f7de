"""The persistent march of the 2D FP32 masked kernel (one cooperative launch
for every step of Scheme 1; tiles wait on the step counters of the 3 x 3
block of tiles around them) through the C ABI.

* against the FP64 oracle over whole marches (max-abs 1e-5), on meshes with
  several tile rows and columns and a ragged last tile, Q = 4, 6, 8 and
  window widths 4..9;
* against the per-step launches of the same plan: the same tile arithmetic,
  so the two agree bit for bit (odd and even step counts, resumed marches,
  random terminal fields, fk_solve's graph path on the 1025 x 513 workload);
* the eligibility rule (no tile shorter than its halo) and the bounded wait:
  one tile that never publishes its step count makes its neighbours' waits
  run out, the device error word reads FK_ERR_TIMEOUT, and the next march on
  the same plan is correct.
"""
import math
import os

import numpy as np
import pytest

import fk_inputs

pytestmark = pytest.mark.gpu
TOL32 = 1e-5
NCPU = os.cpu_count() or 1
FAM = {"const_drift": 0, "cellular_flow": 1}


@pytest.fixture(scope="module")
def fk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_14561_gb300 as fk
    fk.load()
    return fk


def _spec(fk, w):
    return fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"],
                       params=w["params"], q=w["q"], dt=w["dt"], n_steps=w["n_steps"],
                       precision="fp32")


def _plan(fk, monkeypatch, w, mode, tile=None):
    monkeypatch.setenv("FK_STEP_KERNEL", "masked")
    monkeypatch.setenv("FK_MARCH", mode)
    if tile:
        monkeypatch.setenv("FK_STEP_TILE", tile)
    else:
        monkeypatch.delenv("FK_STEP_TILE", raising=False)
    plan = fk.Plan(_spec(fk, w))
    monkeypatch.delenv("FK_MARCH")
    return plan


def _run(plan, fn):
    import torch
    out = fn(plan)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    return out.double().cpu().numpy()


def _both(fk, monkeypatch, w, fn, tile="16,0,2"):
    """fn on a persistent-march plan and on a per-step plan of the same tiles
    (16-row tiles unless given: taller than every halo here)."""
    res = {}
    for mode in ("persistent", "steps"):
        plan = _plan(fk, monkeypatch, w, mode, tile)
        info = plan.info()
        assert info["step_kernel"] == "masked" and info["march_mode"] == mode
        res[mode] = _run(plan, fn)
        plan.close()
    return res, info


def _oracle(oracle, w, n_from, n_to, u_in=None):
    g = oracle.Grid(tuple(w["n"]), tuple(w["lo"]), tuple(w["hi"]))
    return oracle.march(g, FAM[w["family"]], list(w["params"]), w["q"], w["dt"], n_from, n_to,
                        u_in, nthreads=NCPU)


def _cellular(n, q, D, dt, n_steps):
    return fk_inputs.workload("cellular_1025x513", n=n, q=q, n_steps=n_steps, precision="fp32",
                              params=(1.0, 0.2, 2 * math.pi, D), dt=dt)


# (mesh, Q, D, dt, window width W): isotropic meshes on [0,2]x[0,1]; the
# last tile column and row are ragged (interior 159 x 79 = 4 x 32 + 31 columns)
CASES = [
    ((161, 81), 6, 0.025, 1e-3, 6),
    ((161, 81), 8, 0.05, 1e-3, 9),
    ((161, 81), 4, 0.05, 1e-3, 6),
    ((131, 67), 4, 0.02, 1e-3, 4),
]


@pytest.mark.parametrize("n,q,D,dt,W", CASES)
def test_persistent_march_vs_oracle_and_steps(fk, oracle, monkeypatch, n, q, D, dt, W):
    w = _cellular(n, q, D, dt, 101)
    res, info = _both(fk, monkeypatch, w, lambda p: p.solve())
    assert info["window_rows"] == W
    assert np.array_equal(res["persistent"], res["steps"])
    assert np.abs(res["persistent"] - _oracle(oracle, w, w["n_steps"], 0)).max() <= TOL32


@pytest.mark.parametrize("n_from,n_to", [(40, 0), (40, 3), (17, 15), (9, 6)])
def test_persistent_resumed_march_random_field(fk, oracle, monkeypatch, n_from, n_to):
    """fk_march from a random field over odd and even step counts (the last
    step lands in the caller's buffer either way)."""
    import torch
    w = _cellular((161, 81), 6, 0.025, 1e-3, 40)
    u0 = fk_inputs.random_field((81, 161), seed=7)
    t = torch.tensor(u0, dtype=torch.float32, device="cuda")
    res, _ = _both(fk, monkeypatch, w, lambda p: p.march(n_from, n_to, t))
    assert np.array_equal(res["persistent"], res["steps"])
    want = _oracle(oracle, w, n_from, n_to, u0)
    assert np.abs(res["persistent"] - want).max() <= TOL32


def test_persistent_const_drift_in_place(fk, oracle, monkeypatch):
    """A march whose input and output are the same buffer."""
    import torch
    w = _cellular((161, 81), 4, 0.02, 1e-3, 30)
    w.update(family="const_drift", params=(0.7, -0.4, 0.0, 0.02))
    u0 = fk_inputs.random_field((81, 161), seed=5)

    def in_place(p):
        t = torch.tensor(u0, dtype=torch.float32, device="cuda")
        return p.march(30, 0, t, out=t)
    res, _ = _both(fk, monkeypatch, w, in_place)
    assert np.array_equal(res["persistent"], res["steps"])
    assert np.abs(res["persistent"] - _oracle(oracle, w, 30, 0, u0)).max() <= TOL32


def test_persistent_benchmark_workload_graph(fk, monkeypatch):
    """fk_solve (captured graph) on the 1025 x 513 workload, 200 steps from a
    random terminal field, twice on the same plan (graph replay)."""
    import torch
    w = fk_inputs.workload("cellular_1025x513", n_steps=200)
    u0 = torch.tensor(fk_inputs.random_field((513, 1025), seed=2), dtype=torch.float32,
                      device="cuda")

    def twice(p):
        a = p.solve(u0)
        b = p.solve(u0)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        return b
    res, info = _both(fk, monkeypatch, w, twice, tile=None)
    assert np.array_equal(res["persistent"], res["steps"])


def test_persistent_needs_tiles_taller_than_the_halo(fk, monkeypatch):
    """4-row tiles with a 9-wide window (halo 4 rows): the tiles around a
    tile would not cover its staged halo, so the plan keeps per-step
    launches even when the persistent march is asked for."""
    w = _cellular((161, 81), 8, 0.05, 1e-3, 10)
    plan = _plan(fk, monkeypatch, w, "persistent", tile="4,0,2")
    info = plan.info()
    assert info["step_kernel"] == "masked" and info["window_rows"] == 9
    assert info["tile"][1] == 4 and info["march_mode"] == "steps"
    plan.close()


def test_persistent_wait_timeout_is_reported(fk, monkeypatch):
    import torch
    from paper_2104_14561_gb300 import _lib as L
    w = _cellular((161, 81), 6, 0.025, 1e-3, 20)
    plan = _plan(fk, monkeypatch, w, "persistent", tile="16,0,2")
    assert plan.info()["march_mode"] == "persistent"
    u0 = torch.tensor(fk_inputs.random_field((81, 161), seed=9), dtype=torch.float32,
                      device="cuda")
    monkeypatch.setenv("FK_TEST_STALL_MARCH", "1")
    plan.march(20, 0, u0)
    torch.cuda.synchronize()
    monkeypatch.delenv("FK_TEST_STALL_MARCH")
    assert L.STATUS[plan.last_device_error()] == "FK_ERR_TIMEOUT"
    # the context is still usable and the next march is correct
    got = _run(plan, lambda p: p.march(20, 0, u0))
    plan.close()
    ref = _plan(fk, monkeypatch, w, "steps", tile="16,0,2")
    want = _run(ref, lambda p: p.march(20, 0, u0))
    ref.close()
    assert np.array_equal(got, want)
