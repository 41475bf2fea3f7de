"""Non-uniform axes in d = 3 on the GPU (Sec. 3.1.2 per direction; the
radial grid of the runaway-electron study of Sec. 4.3), through the C ABI,
against the FP64 oracle on the same axes and seeded inputs.  Tolerances
(max-abs): 1e-12 FP64, 1e-5 FP32.

* constant drift in a box with all three axes graded towards their faces
  (whole marches, FP64 and FP32);
* explicit uniform coordinates agree with the uniform plan (different
  arithmetic: physical positions, walked cells and per-cell widths instead
  of index space);
* the runaway model on the paper's two-spacing radial grid (coarse on
  [0, r_D], fine on [r_D, 1]) on a small mesh: whole marches (FP64, FP32)
  and every horizon of Algorithm 1;
* the full-size non-uniform runaway workload over one step at sampled nodes.
"""
import os

import numpy as np
import pytest

import fk_inputs

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1
RUNAWAY = fk_inputs.workload("runaway_97x65x41")["params"]


@pytest.fixture(scope="module")
def fk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_14561_gb300 as fk
    fk.load()
    return fk


def _spec(fk, w, axes=True):
    return fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"], params=w["params"],
                       q=w["q"], dt=w["dt"], n_steps=w["n_steps"], precision=w["precision"],
                       axes=w["axes"] if axes else None)


def _family(oracle, w):
    return {"const_drift": oracle.CONST_DRIFT, "runaway": oracle.RUNAWAY}[w["family"]]


def _oracle(oracle, w, k=None, u0=None):
    g = oracle.Grid(tuple(w["n"]), tuple(w["lo"]), tuple(w["hi"]), 0, w["axes"])
    return oracle.march(g, _family(oracle, w), list(w["params"]), w["q"], w["dt"],
                        k or w["n_steps"], 0, u0, nthreads=NCPU)


def _solve(fk, w, axes=True):
    import torch
    plan = fk.Plan(_spec(fk, w, axes))
    out = plan.solve()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    info = plan.info()
    plan.close()
    return out.double().cpu().numpy(), info


def _box(precision, n_steps=15):
    axes = tuple(fk_inputs.graded_axis(-1.0, 1.0, n, s) for n, s in ((21, 0.4), (17, 0.3), (13, 0.5)))
    return dict(n=(21, 17, 13), lo=(-1.0,) * 3, hi=(1.0,) * 3, family="const_drift",
                params=(0.3, -0.2, 0.1, 0.4), q=4, dt=2e-3, n_steps=n_steps,
                precision=precision, axes=axes)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_graded_box_const_drift(fk, oracle, precision, tol):
    w = _box(precision)
    got, info = _solve(fk, w)
    assert info["nonuniform"] and info["step_kernel"] == "window3d"
    assert np.abs(got - _oracle(oracle, w)).max() <= tol


def test_explicit_uniform_axes_match_uniform_plan(fk):
    for family, params, lo, hi in (("const_drift", (0.3, -0.2, 0.1, 0.4), (-1.0,) * 3, (1.0,) * 3),
                                   ("runaway", RUNAWAY, (2.0, -1.0, 0.0), (12.0, 1.0, 1.0))):
        n = (21, 17, 11)
        axes = tuple(np.linspace(lo[m], hi[m], n[m]) for m in range(3))
        w = dict(n=n, lo=lo, hi=hi, family=family, params=params, q=4, dt=0.01 if
                 family == "runaway" else 2e-3, n_steps=10, precision="fp64", axes=axes)
        nu, info = _solve(fk, w)
        un, _ = _solve(fk, w, axes=False)
        assert info["nonuniform"]
        assert np.abs(nu - un).max() <= 1e-12, family


def _runaway_small(precision, n_steps=12):
    r = fk_inputs.two_spacing_axis(0.0, 0.7, 1.0, 0.1, 0.025)
    return dict(n=(13, 9, len(r)), lo=(2.0, -1.0, 0.0), hi=(12.0, 1.0, 1.0), family="runaway",
                params=RUNAWAY, q=4, dt=0.05, n_steps=n_steps, precision=precision,
                axes=(None, None, r))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_runaway_two_spacing_radial_grid(fk, oracle, precision, tol):
    w = _runaway_small(precision)
    got, info = _solve(fk, w)
    assert info["nonuniform"]
    want = _oracle(oracle, w)
    assert want[:, :, :-1].max() > 1e-3  # a runaway probability off the p_max face
    assert np.abs(got - want).max() <= tol


def test_runaway_two_spacing_horizons(fk, oracle):
    import torch
    w = _runaway_small("fp64", n_steps=6)
    plan = fk.Plan(_spec(fk, w))
    hz = plan.solve_horizons()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    hz = hz.cpu().numpy()
    plan.close()
    for k in (1, 3, 6):
        assert np.abs(hz[k - 1] - _oracle(oracle, w, k)).max() <= 1e-12, k


def test_runaway_nonuniform_workload_sampled_step(fk, oracle):
    """The 97 x 65 x 128 workload on the paper's radial grid (FP32): one step
    from a random field at sampled nodes (every face included) against the
    oracle's step there."""
    import torch
    w = fk_inputs.workload("runaway_nonuniform_97x65x128")
    shape = tuple(reversed(w["n"]))
    plan = fk.Plan(_spec(fk, w))
    assert plan.info()["nonuniform"] and plan.info()["window_rows"] <= 8
    u1 = fk_inputs.random_field(shape, seed=83, boundary_one=False)
    n = 100
    got = plan.march(n + 1, n, torch.tensor(u1, dtype=torch.float32, device="cuda"))
    got = got.double().cpu().numpy().reshape(-1)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    plan.close()
    nodes = fk_inputs.sample_nodes(shape, 3000, seed=19)
    g = oracle.Grid(tuple(w["n"]), tuple(w["lo"]), tuple(w["hi"]), 0, fk_inputs.axes_of(w))
    want = oracle.step_nodes(g, oracle.RUNAWAY, list(w["params"]), w["q"], w["dt"], n, u1, nodes,
                             nthreads=NCPU)
    assert np.abs(got[nodes] - want).max() <= 1e-5
