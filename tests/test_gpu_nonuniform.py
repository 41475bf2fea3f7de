"""Non-uniform axes on the GPU (the mesh of Sec. 3.1.2, graded as in the
paper's Sec. 4.3 study), through the C ABI, against the FP64 oracle on the
same axes and seeded inputs.  Tolerances (max-abs): 1e-12 FP64, 1e-5 FP32.

* both axes graded towards their faces (cellular flow, FP64 and FP32);
* a two-spacing axis (coarse, then 20x finer next to one face), the mesh
  shape of the paper's non-uniform runaway-electron grid;
* explicit uniform coordinates agree with the uniform plan (different
  arithmetic: physical positions and cell search instead of index space);
* every horizon of Algorithm 1 on a graded mesh;
* a random terminal field and the paper's own flow family.
"""
import math
import os

import numpy as np
import pytest

import fk_inputs

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1
CELL = (1.0, 0.3, 2 * math.pi, 2e-3)


@pytest.fixture(scope="module")
def fk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_14561_gb300 as fk
    fk.load()
    return fk


graded = fk_inputs.graded_axis


def two_spacing(lo, mid, hi, coarse, fine):
    a = np.arange(lo, mid - 1e-12, coarse)
    b = mid + np.arange(0, int(round((hi - mid) / fine)) + 1) * fine
    x = np.concatenate([a, b])
    x[-1] = hi
    return x


def _w(axes, precision="fp64", family="cellular_flow", params=CELL, q=4, dt=1e-3, n_steps=20,
       lo=(0.0, 0.0), hi=(2.0, 1.0)):
    return dict(n=(len(axes[0]), len(axes[1])), lo=lo, hi=hi, family=family, params=params,
                q=q, dt=dt, n_steps=n_steps, precision=precision, axes=axes)


def _spec(fk, w, axes=True):
    return fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"], params=w["params"],
                       q=w["q"], dt=w["dt"], n_steps=w["n_steps"], precision=w["precision"],
                       axes=w["axes"] if axes else None)


def _solve(fk, w, u0=None, axes=True):
    import torch
    plan = fk.Plan(_spec(fk, w, axes))
    ut = None if u0 is None else torch.tensor(u0, dtype=plan.dtype, device="cuda")
    out = plan.solve(ut)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    info = plan.info()
    res = out.double().cpu().numpy()
    plan.close()
    return res, info


def _oracle(oracle, w, k=None, u0=None):
    fam = {"cellular_flow": oracle.CELLULAR_FLOW, "paper_cellular": oracle.PAPER_CELLULAR,
           "const_drift": oracle.CONST_DRIFT}[w["family"]]
    g = oracle.Grid(tuple(w["n"]), tuple(w["lo"]), tuple(w["hi"]), axes=tuple(w["axes"]))
    return oracle.march(g, fam, list(w["params"]), w["q"], w["dt"], k or w["n_steps"], 0, u0,
                        nthreads=NCPU)


@pytest.mark.parametrize("precision,q,tol", [("fp64", 4, 1e-12), ("fp32", 6, 1e-5)])
def test_graded_both_axes(fk, oracle, precision, q, tol):
    w = _w((graded(0.0, 2.0, 61, 0.8), graded(0.0, 1.0, 41, 0.6)), precision=precision, q=q)
    got, info = _solve(fk, w)
    assert info["step_kernel"] == "direct" and info["nonuniform"] and not info["periodic_x"]
    assert np.abs(got - _oracle(oracle, w)).max() <= tol
    assert got[1:-1, 1:-1].max() > 0.05


def test_two_spacing_axis(fk, oracle):
    ay = two_spacing(0.0, 0.7, 1.0, 0.05, 0.0025)
    w = _w((np.linspace(0.0, 2.0, 49), ay), params=(1.0, 0.3, 2 * math.pi, 1e-4), q=6,
           n_steps=15)
    got, _ = _solve(fk, w)
    assert np.abs(got - _oracle(oracle, w)).max() <= 1e-12


def test_explicit_uniform_axes_match_uniform_plan(fk):
    n = (65, 33)
    ax = (np.linspace(0.0, 2.0, n[0]), np.linspace(0.0, 1.0, n[1]))
    w = _w(ax, n_steps=30)
    nu, _ = _solve(fk, w)
    un, _ = _solve(fk, w, axes=False)
    assert np.abs(nu - un).max() <= 1e-12


def test_graded_random_field_paper_family(fk, oracle):
    ax = (graded(-math.pi, math.pi, 57, 0.5), graded(0.0, 1.0, 33, 0.7))
    w = _w(ax, family="paper_cellular", params=(10.0, 2.0, 0.15, 2 * math.pi / 10), dt=2e-4,
           lo=(-math.pi, 0.0), hi=(math.pi, 1.0), n_steps=12)
    u0 = fk_inputs.random_field((33, 57), seed=51)
    got, _ = _solve(fk, w, u0)
    assert np.abs(got - _oracle(oracle, w, u0=u0)).max() <= 1e-12


def test_graded_horizons(fk, oracle):
    import torch
    w = _w((graded(0.0, 2.0, 45, 0.8), graded(0.0, 1.0, 29, 0.6)), n_steps=6)
    plan = fk.Plan(_spec(fk, w))
    out = plan.solve_horizons()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    plan.close()
    for k in (1, 3, 6):
        assert np.abs(got[k - 1] - _oracle(oracle, w, k)).max() <= 1e-12, k


def test_graded_batched_equals_single(fk):
    import torch
    ws = [_w((graded(0.0, 2.0, 45, 0.8), graded(0.0, 1.0, 29, 0.6)), precision="fp32"),
          _w((graded(0.0, 2.0, 61, 0.5), graded(0.0, 1.0, 33, 0.5)), precision="fp32")]
    singles = [_solve(fk, w)[0] for w in ws]
    plans = [fk.Plan(_spec(fk, w)) for w in ws]
    outs = fk.solve_batched(plans)
    torch.cuda.synchronize()
    for o, s in zip(outs, singles):
        assert np.array_equal(o.double().cpu().numpy(), s)
    for p in plans:
        p.close()


def test_graded_workload_sampled_step(fk, oracle):
    """The graded benchmark workload (1025 x 513, 6 x 6 points, FP32): one
    step from a random field at sampled nodes against the oracle's step."""
    import torch
    w = fk_inputs.workload("graded_1025x513")
    axes = fk_inputs.axes_of(w)
    ny, nx = w["n"][1], w["n"][0]
    plan = fk.Plan(fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"],
                               params=w["params"], q=w["q"], dt=w["dt"], n_steps=w["n_steps"],
                               precision="fp32", axes=axes))
    u1 = fk_inputs.random_field((ny, nx), seed=53)
    n = 1234
    got = plan.march(n + 1, n, torch.tensor(u1, dtype=torch.float32, device="cuda"))
    got = got.double().cpu().numpy().reshape(-1)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    plan.close()
    nodes = fk_inputs.sample_nodes((ny, nx), 2000, seed=7)
    g = oracle.Grid(tuple(w["n"]), tuple(w["lo"]), tuple(w["hi"]), axes=axes)
    want = oracle.step_nodes(g, oracle.CELLULAR_FLOW, list(w["params"]), w["q"], w["dt"], n, u1,
                             nodes, nthreads=NCPU)
    assert np.abs(got[nodes] - want).max() <= 1e-5


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_graded_1d(fk, oracle, precision, tol):
    """1D drifted Brownian motion (b = 0.5, sigma = 1 on (-1, 1)) on a mesh
    graded towards both faces: the per-step 1D kernel against the oracle,
    every horizon included."""
    import torch
    ax = graded(-1.0, 1.0, 121, 0.6)
    spec = fk.PlanSpec(n=(121,), lo=(-1.0,), hi=(1.0,), family="const_drift",
                       params=(0.5, 0.0, 0.0, 1.0), q=8, dt=1e-3, n_steps=60,
                       precision=precision, axes=(ax,))
    plan = fk.Plan(spec)
    assert plan.info()["nonuniform"] and plan.info()["step_kernel"] == "direct"
    got = plan.solve().double().cpu().numpy()
    hz = plan.solve_horizons().double().cpu().numpy()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    plan.close()
    g = oracle.Grid((121,), (-1.0,), (1.0,), axes=(ax,))
    want = oracle.march(g, oracle.CONST_DRIFT, [0.5, 0.0, 0.0, 1.0], 8, 1e-3, 60, 0)
    assert np.abs(got - want).max() <= tol
    for k in (1, 30):
        wk = oracle.march(g, oracle.CONST_DRIFT, [0.5, 0.0, 0.0, 1.0], 8, 1e-3, k, 0)
        assert np.abs(hz[k - 1] - wk).max() <= tol, k
    assert np.abs(hz[-1] - got).max() <= tol


def test_graded_workload_full_march_vs_golden(fk):
    """The graded benchmark workload: all 2000 FP32 steps against the FP64
    oracle's u^0 at 20k+ sampled nodes (every node next to the boundary
    included), written by tests/golden/make_oracle_golden.py."""
    import torch
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden",
                                "graded_1025x513_oracle_u0.npz"))
    w = fk_inputs.workload("graded_1025x513")
    assert tuple(gold["n"]) == tuple(w["n"]) and int(gold["n_steps"]) == w["n_steps"]
    plan = fk.Plan(fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"],
                               params=w["params"], q=w["q"], dt=w["dt"], n_steps=w["n_steps"],
                               precision="fp32", axes=fk_inputs.axes_of(w)))
    out = plan.solve()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    got = out.double().reshape(-1).cpu().numpy()[gold["nodes"]]
    plan.close()
    err = np.abs(got - gold["u0"]).max()
    print(f"graded_1025x513 fp32 vs fp64 oracle, 2000 steps: max-abs {err:.3e}")
    assert err <= 1e-5
