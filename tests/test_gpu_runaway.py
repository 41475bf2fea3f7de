"""The runaway-electron model of Sec. 4.3 (Eq. (ex32d), d = 3, x = (p, xi,
r)) on the GPU, through the C ABI, against the FP64 oracle on the same
seeded inputs.  Tolerances (max-abs): 1e-12 FP64, 1e-5 FP32.

* whole marches on small meshes at the paper's parameters and at a set with
  a strong field, radiation and radial transport (every face rule at work:
  runaway exit at p_max, value 0 at p_min and at the wall, mirrors at
  xi = +-1 and r = 0);
* one step from a random field (every face's nodes included);
* every horizon (Algorithm 1) from the runaway indicator;
* the 97 x 65 x 41 benchmark workload over one step at sampled nodes;
* the thermal-quench variant: whole marches at a strong-field test set and
  at the constants the paper prints for it (p up to 50), every horizon, and
  one late step of its 97 x 33 x 41 workload at sampled nodes.
"""
import os

import numpy as np
import pytest

import fk_inputs

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1
PAPER = (0.3, 1e5, 1.0, 0.042, 1.0, 1.0, 0.7, 1e-2, 20.0, 0.003, 1e-4)
STRONG = (3.0, 50.0, 1.0, 0.042, 1.0, 1.0, 0.5, 0.05, 20.0, 0.05, 0.02)


@pytest.fixture(scope="module")
def fk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_14561_gb300 as fk
    fk.load()
    return fk


def _w(n, params, hi_p, dt, n_steps, precision="fp64", q=4):
    return dict(n=n, lo=(2.0, -1.0, 0.0), hi=(hi_p, 1.0, 1.0), family="runaway",
                params=params, q=q, dt=dt, n_steps=n_steps, precision=precision)


def _spec(fk, w):
    return fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family="runaway", params=w["params"],
                       q=w["q"], dt=w["dt"], n_steps=w["n_steps"], precision=w["precision"])


def _grid(oracle, w):
    return oracle.Grid(tuple(w["n"]), tuple(w["lo"]), tuple(w["hi"]))


def _oracle(oracle, w, k=None, u0=None):
    return oracle.march(_grid(oracle, w), oracle.RUNAWAY, list(w["params"]), w["q"], w["dt"],
                        k or w["n_steps"], 0, u0, nthreads=NCPU)


def _solve(fk, w, u0=None):
    import torch
    plan = fk.Plan(_spec(fk, w))
    ut = None if u0 is None else torch.tensor(u0, dtype=plan.dtype, device="cuda")
    out = plan.solve(ut)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    info = plan.info()
    res = out.double().cpu().numpy()
    plan.close()
    return res, info


@pytest.mark.parametrize("case", ["paper", "strong"])
def test_runaway_fp64_vs_oracle(fk, oracle, case):
    if case == "paper":
        w = _w((25, 17, 13), PAPER, 50.0, 0.02, 25)
    else:
        w = _w((21, 17, 11), STRONG, 12.0, 0.02, 40)
    got, info = _solve(fk, w)
    assert info["step_kernel"] == "window3d"
    want = _oracle(oracle, w)
    assert np.abs(got - want).max() <= 1e-12
    assert got[..., -1].min() == 1.0 and got[..., 0].max() == 0.0
    if case == "strong":  # T = 0.8 carried a runaway front into the box (129 nodes)
        inner = got[1:-1, 1:-1, 1:-1]
        assert np.count_nonzero((inner > 0.05) & (inner < 0.95)) > 50


def test_runaway_fp32_random_field_step(fk, oracle):
    w = _w((21, 17, 11), STRONG, 12.0, 0.05, 3, precision="fp32")
    u1 = fk_inputs.random_field((11, 17, 21), seed=71, boundary_one=False)
    got, _ = _solve(fk, w, u1)
    assert np.abs(got - _oracle(oracle, w, u0=u1)).max() <= 1e-5


def test_runaway_fp64_random_field_one_step(fk, oracle):
    import torch
    w = _w((21, 17, 11), STRONG[:9] + (0.05, 0.3), 12.0, 0.02, 2)
    u1 = fk_inputs.random_field((11, 17, 21), seed=72, boundary_one=False)
    plan = fk.Plan(_spec(fk, w))
    got = plan.march(1, 0, torch.tensor(u1, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    plan.close()
    want = oracle.march(_grid(oracle, w), oracle.RUNAWAY, list(w["params"]), 4, w["dt"], 1, 0, u1)
    assert np.abs(got.cpu().numpy() - want).max() <= 1e-12


def test_runaway_horizons(fk, oracle):
    import torch
    w = _w((21, 17, 11), STRONG, 12.0, 0.05, 5)
    plan = fk.Plan(_spec(fk, w))
    hz = plan.solve_horizons()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    hz = hz.cpu().numpy()
    plan.close()
    for k in (1, 3, 5):
        assert np.abs(hz[k - 1] - _oracle(oracle, w, k)).max() <= 1e-12, k


def test_runaway_workload_sampled_step(fk, oracle):
    """The 97 x 65 x 41 workload at the paper's parameters (FP32, 4^3
    points): one step from a random field at sampled nodes (every face
    included) against the oracle's step there."""
    import torch
    w = fk_inputs.workload("runaway_97x65x41")
    shape = tuple(reversed(w["n"]))
    plan = fk.Plan(_spec(fk, w))
    assert plan.info()["window_rows"] <= 8
    u1 = fk_inputs.random_field(shape, seed=73, boundary_one=False)
    n = 100
    got = plan.march(n + 1, n, torch.tensor(u1, dtype=torch.float32, device="cuda"))
    got = got.double().cpu().numpy().reshape(-1)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    plan.close()
    nodes = fk_inputs.sample_nodes(shape, 3000, seed=13)
    want = oracle.step_nodes(_grid(oracle, w), oracle.RUNAWAY, list(w["params"]), w["q"],
                             w["dt"], n, u1, nodes, nthreads=NCPU)
    assert np.abs(got[nodes] - want).max() <= 1e-5


# the thermal-quench variant (end of Sec. 4.3): the paper's constants with
# E_0 = 0.1 and t_star = 0.5, on p in (2, 8), so that the field grows and
# the collisions with it over the march
QUENCH = (0.1, 6000.0, 1.0, 3.0, 0.005, 3.0, 0.5, 0.0, 1e-4, 2.0, 0.0, 0.01, 511.0)


def _wq(precision="fp64", n_steps=25):
    return dict(n=(21, 17, 11), lo=(2.0, -1.0, 0.0), hi=(8.0, 1.0, 1.0),
                family="runaway_quench", params=QUENCH, q=4, dt=0.02, n_steps=n_steps,
                precision=precision)


def _spec_q(fk, w):
    return fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family="runaway_quench",
                       params=w["params"], q=w["q"], dt=w["dt"], n_steps=w["n_steps"],
                       precision=w["precision"])


def _oracle_q(oracle, w, k=None):
    return oracle.march(_grid(oracle, w), oracle.RUNAWAY_QUENCH, list(w["params"]), w["q"],
                        w["dt"], k or w["n_steps"], 0, nthreads=NCPU)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_quench_vs_oracle(fk, oracle, precision, tol):
    import torch
    w = _wq(precision)
    plan = fk.Plan(_spec_q(fk, w))
    got = plan.solve().double().cpu().numpy()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    plan.close()
    assert np.abs(got - _oracle_q(oracle, w)).max() <= tol


def test_quench_horizons(fk, oracle):
    """Every horizon of the non-autonomous model (Algorithm 1): horizon k
    marches k steps with the constants of t_{k-1}, ..., t_0."""
    import torch
    w = _wq(n_steps=12)
    plan = fk.Plan(_spec_q(fk, w))
    hz = plan.solve_horizons()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    hz = hz.cpu().numpy()
    plan.close()
    for k in (1, 6, 12):
        assert np.abs(hz[k - 1] - _oracle_q(oracle, w, k)).max() <= 1e-12, k


# the constants the paper prints for the quench (E_0 = 1e-3, tau = 6000,
# r_D = 0, W = 1e-4, Delta_p = 2, V_0 = 0), D_0 = 0.01, t_star = 2
QUENCH_PAPER = fk_inputs.workload("runaway_quench_97x33x41")["params"]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_quench_paper_parameters_vs_oracle(fk, oracle, precision, tol):
    """A whole march to T = 10 at the paper's quench constants on p in (2,
    50): the temperature falls from 3 keV to about 25 eV and the field grows
    from 1e-3 to about 1.3, so that a runaway probability spreads from the
    p_max face into the interior."""
    import torch
    w = dict(n=(25, 9, 11), lo=(2.0, -1.0, 0.0), hi=(50.0, 1.0, 1.0), family="runaway_quench",
             params=QUENCH_PAPER, q=4, dt=0.01, n_steps=1000, precision=precision)
    plan = fk.Plan(_spec_q(fk, w))
    got = plan.solve().double().cpu().numpy()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    plan.close()
    want = _oracle_q(oracle, w)
    assert want[:, :, :-1].max() > 1e-3  # off the p_max face
    assert np.abs(got - want).max() <= tol


def test_quench_workload_sampled_late_step(fk, oracle):
    """The 97 x 33 x 41 quench workload (FP32): one step at n = 8000 (t =
    8, about 35 eV) from a random field, at sampled nodes against the
    oracle's step there."""
    import torch
    w = fk_inputs.workload("runaway_quench_97x33x41")
    shape = tuple(reversed(w["n"]))
    plan = fk.Plan(_spec_q(fk, w))
    assert plan.info()["window_rows"] <= 8
    u1 = fk_inputs.random_field(shape, seed=79, boundary_one=False)
    n = 8000
    got = plan.march(n + 1, n, torch.tensor(u1, dtype=torch.float32, device="cuda"))
    got = got.double().cpu().numpy().reshape(-1)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    plan.close()
    nodes = fk_inputs.sample_nodes(shape, 3000, seed=17)
    want = oracle.step_nodes(_grid(oracle, w), oracle.RUNAWAY_QUENCH, list(w["params"]), w["q"],
                             w["dt"], n, u1, nodes, nthreads=NCPU)
    assert np.abs(got[nodes] - want).max() <= 1e-5
