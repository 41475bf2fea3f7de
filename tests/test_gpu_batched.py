"""GPU checks of the batched march (fk_solve_batched) of many independent
instances (uneven meshes and coefficients), with each of its two
strategies: one cooperative persistent launch through all time steps, and
the instances' own graph marches on concurrent side streams.

* every instance equals its own single-plan fk_solve (FP64 to 1e-14, FP32
  to 1e-6) and, for small FP64 instances, the oracle (1e-12);
* terminal fields given per instance, including one aliased with its output;
* the 64-instance sweep's meshes and coefficients (fewer steps) against the
  single-plan march, and the whole 1000-step sweep's three smallest
  instances against the FP64 oracle (1e-5);
* the bounded grid barrier: with a phantom CTA that never arrives every wait
  runs into its 1 s limit, the launch ends, the host reads FK_ERR_TIMEOUT,
  and the context stays usable.
"""
import math
import os

import numpy as np
import pytest

import fk_inputs

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module")
def fk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_14561_gb300 as fk
    fk.load()
    return fk


@pytest.fixture(params=["persistent", "streams"])
def batch_mode(request, monkeypatch):
    """The strategy fk_solve_batched uses in the test."""
    monkeypatch.setenv("FK_BATCH_MODE", request.param)
    return request.param


def _plan(fk, w, **kw):
    d = dict(w)
    d.update(kw)
    return fk.Plan(fk.PlanSpec(n=d["n"], lo=d["lo"], hi=d["hi"], family=d["family"],
                               params=d["params"], q=d["q"], dt=d["dt"], n_steps=d["n_steps"],
                               precision=d["precision"], path="matrix_free"))


def _mixed(precision, n_steps=25, q=6):
    rng = np.random.default_rng(4)
    ws = []
    for nx, ny in ((67, 35), (130, 41), (33, 33), (257, 129), (3, 9), (95, 48)):
        D = 10 ** rng.uniform(-3, -1.5)
        A = rng.uniform(0.5, 2.0)
        ws.append(dict(n=(nx, ny), lo=(0.0, 0.0), hi=(2.0, 1.0), family="cellular_flow",
                       params=(A, 0.2, 2 * math.pi, D), q=q, dt=1e-3, n_steps=n_steps,
                       precision=precision))
    ws.append(dict(n=(50, 30), lo=(-1.0, -1.0), hi=(1.0, 1.0), family="const_drift",
                   params=(0.5, -0.3, 0.0, 0.4), q=q, dt=1e-3, n_steps=n_steps,
                   precision=precision))
    return ws


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-14), ("fp32", 1e-6)])
def test_batched_equals_single_plans(fk, precision, tol, batch_mode):
    import torch
    ws = _mixed(precision)
    plans = [_plan(fk, w) for w in ws]
    outs = fk.solve_batched(plans)
    torch.cuda.synchronize()
    assert plans[0].info()["batch_mode"] == batch_mode
    assert plans[0].last_device_error() == 0
    for p, o in zip(plans, outs):
        ref = p.solve()
        torch.cuda.synchronize()
        assert (o - ref).abs().max().item() <= tol
    # a second call reuses the cached graph
    outs2 = fk.solve_batched(plans)
    torch.cuda.synchronize()
    for o, o2 in zip(outs, outs2):
        assert torch.equal(o, o2)
    for p in plans:
        p.close()


def test_batched_fp64_vs_oracle(fk, oracle, batch_mode):
    import torch
    ws = _mixed("fp64", n_steps=12)[:4]
    plans = [_plan(fk, w) for w in ws]
    outs = fk.solve_batched(plans)
    torch.cuda.synchronize()
    assert plans[0].info()["batch_mode"] == batch_mode
    for w, o in zip(ws, outs):
        g = oracle.Grid(w["n"], w["lo"], w["hi"])
        want = oracle.march(g, 1, list(w["params"]), w["q"], w["dt"], w["n_steps"], 0,
                            nthreads=NCPU)
        assert np.abs(o.cpu().numpy() - want).max() <= 1e-12
    for p in plans:
        p.close()


@pytest.mark.parametrize("n_steps", [7, 8])
def test_batched_terminal_fields_and_aliasing(fk, n_steps, batch_mode):
    import torch
    ws = _mixed("fp64", n_steps=n_steps)[:3]
    plans = [_plan(fk, w) for w in ws]
    u0 = [torch.tensor(fk_inputs.random_field(p.shape, seed=s), dtype=torch.float64,
                       device="cuda") for s, p in enumerate(plans)]
    refs = [p.solve(u.clone()) for p, u in zip(plans, u0)]
    outs = [p.empty() for p in plans]
    ins = [u0[0], None, u0[2].clone()]
    outs[2] = ins[2]  # in place for the third instance
    fk.solve_batched(plans, ins, outs)
    torch.cuda.synchronize()
    assert plans[0].info()["batch_mode"] == batch_mode
    chi_ref = plans[1].solve()
    torch.cuda.synchronize()
    assert (outs[0] - refs[0]).abs().max().item() <= 1e-14
    assert (outs[1] - chi_ref).abs().max().item() <= 1e-14
    assert (outs[2] - refs[2]).abs().max().item() <= 1e-14
    for p in plans:
        p.close()


def test_batched_sweep_instances(fk, batch_mode):
    import torch
    ws = [dict(w, n_steps=20) for w in fk_inputs.batched_instances()]
    plans = [_plan(fk, w) for w in ws]
    outs = fk.solve_batched(plans)
    torch.cuda.synchronize()
    assert plans[0].info()["batch_mode"] == batch_mode
    assert all(p.last_device_error() == 0 for p in plans)
    worst = 0.0
    for p, o in zip(plans, outs):
        ref = p.solve()
        torch.cuda.synchronize()
        worst = max(worst, (o - ref).abs().max().item())
        p.close()
    assert worst <= 1e-6


@pytest.fixture(scope="module")
def sweep_oracle(oracle):
    """The FP64 oracle's full 1000-step marches of the sweep's three
    smallest instances (279 x 140 to 311 x 156 nodes), by instance index."""
    ws = fk_inputs.batched_instances()
    small = sorted(range(len(ws)), key=lambda m: ws[m]["n"][0] * ws[m]["n"][1])[:3]
    out = {}
    for m in small:
        w = ws[m]
        g = oracle.Grid(w["n"], w["lo"], w["hi"])
        out[m] = oracle.march(g, 1, list(w["params"]), w["q"], w["dt"], w["n_steps"], 0,
                              nthreads=NCPU)
    return out


def test_batched_sweep_full_march_vs_oracle(fk, sweep_oracle, batch_mode):
    """The 64-instance sweep itself (1000 FP32 steps, every instance in one
    batched call): its three smallest instances against the FP64 oracle's
    whole marches, max-abs 1e-5 over every node."""
    import torch
    ws = fk_inputs.batched_instances()
    plans = [_plan(fk, w) for w in ws]
    outs = fk.solve_batched(plans)
    torch.cuda.synchronize()
    assert plans[0].info()["batch_mode"] == batch_mode
    assert all(p.last_device_error() == 0 for p in plans)
    for m, want in sweep_oracle.items():
        err = np.abs(outs[m].double().cpu().numpy() - want).max()
        assert err <= 1e-5, (m, ws[m]["n"], err)
    for p in plans:
        p.close()


def test_barrier_timeout_is_reported(fk, monkeypatch):
    import torch
    from paper_2104_14561_gb300 import _lib as L
    monkeypatch.setenv("FK_BATCH_MODE", "persistent")
    ws = _mixed("fp32", n_steps=3)[:2]
    plans = [_plan(fk, w) for w in ws]
    os.environ["FK_TEST_STALL_BARRIER"] = "1"
    try:
        fk.solve_batched(plans)
        torch.cuda.synchronize()
    finally:
        del os.environ["FK_TEST_STALL_BARRIER"]
    assert plans[0].info()["batch_mode"] == "persistent"
    assert L.STATUS[plans[0].last_device_error()] == "FK_ERR_TIMEOUT"
    # the context is still usable and the next batch is correct
    outs = fk.solve_batched(plans)
    torch.cuda.synchronize()
    assert plans[0].last_device_error() == 0
    for p, o in zip(plans, outs):
        assert (o - p.solve()).abs().max().item() <= 1e-6
        p.close()
