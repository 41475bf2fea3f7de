"""GPU adjoint (fk_adjoint) of the march: dL/dtheta and dL/du^N for
L = <g, u^0>, checked against
* the FP64 CPU oracle adjoint (FP64 plan: 1e-10 relative on parameters,
  1e-12 absolute on the terminal field; FP32 plan: 1e-3 relative, reported);
* its own results at other checkpoint intervals K (recompute is exact);
* central finite differences of FP64 GPU marches at the full-size adjoint
  workload (1025 x 513, 6 x 6 points, 2000 steps): h = 1e-4 for A and eps,
  1e-4 D for D, objective L = mean of u^0 over interior nodes;
* the FP32 march's adjoint against the FP64 one at that size (1e-3 gate on
  the parameters; 5e-3 relative L2 on the terminal-field gradient, which
  measures 1.7e-3 from a random smooth terminal field);
* the torch.autograd.Function wrapper.
"""
import math
import os

import numpy as np
import pytest

import fk_inputs

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1
SMALL = dict(n=(41, 21), lo=(0.0, 0.0), hi=(2.0, 1.0), family="cellular_flow",
             params=(1.0, 0.3, 2 * math.pi, 0.02), q=4, dt=2e-3, n_steps=15)


@pytest.fixture(scope="module")
def fk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_14561_gb300 as fk
    fk.load()
    return fk


def _spec(fk, w, precision):
    return fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"],
                       params=w["params"], q=w["q"], dt=w["dt"], n_steps=w["n_steps"],
                       precision=precision)


def _gpu_adjoint(fk, w, precision, cot, u0=None, K=50, kernel=None):
    import torch
    plan = fk.Plan(_spec(fk, w, precision))
    ut = None if u0 is None else torch.tensor(u0, dtype=plan.dtype, device="cuda")
    g = torch.tensor(cot, dtype=torch.float64, device="cuda")
    dth, du = plan.adjoint(g, ut, checkpoint_every=K)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    if kernel is not None:
        assert plan.info()["adjoint_kernel"] == kernel
    r = dth.cpu().numpy(), du.double().cpu().numpy()
    plan.close()
    return r


@pytest.mark.parametrize("family", ["cellular_flow", "const_drift"])
def test_adjoint_fp64_vs_oracle(fk, oracle, family):
    w = dict(SMALL)
    if family == "const_drift":
        w.update(family="const_drift", params=(0.6, -0.4, 0.0, 0.35), lo=(-1.0, -1.0),
                 hi=(1.0, 1.0), n=(31, 25))
    shape = (w["n"][1], w["n"][0])
    cot = np.random.default_rng(1).standard_normal(shape)
    u0 = fk_inputs.random_field(shape, seed=3)
    dth, du = _gpu_adjoint(fk, w, "fp64", cot, u0, K=4)
    g = oracle.Grid(w["n"], w["lo"], w["hi"])
    fam = oracle.CELLULAR_FLOW if family == "cellular_flow" else oracle.CONST_DRIFT
    odth, odu = oracle.adjoint(g, fam, list(w["params"]), w["q"], w["dt"], w["n_steps"], cot, u0)
    np.testing.assert_allclose(dth, odth, rtol=1e-10, atol=1e-12)
    assert np.abs(du - odu).max() <= 1e-12


@pytest.mark.parametrize("n", [(3, 3), (5, 3), (3, 6), (4, 4)])
def test_adjoint_fp64_tiny_meshes_vs_oracle(fk, oracle, n):
    """Meshes with 3 or 4 nodes on an axis, where the end rule of the slopes
    (node 0 takes node 1's slope, node n-1 that of node n-2) puts both ends'
    slopes on the same interior stencil."""
    w = dict(SMALL, n=n, n_steps=6)
    shape = (n[1], n[0])
    cot = np.random.default_rng(5).standard_normal(shape)
    u0 = fk_inputs.random_field(shape, seed=7)
    dth, du = _gpu_adjoint(fk, w, "fp64", cot, u0, K=2)
    g = oracle.Grid(w["n"], w["lo"], w["hi"])
    odth, odu = oracle.adjoint(g, oracle.CELLULAR_FLOW, list(w["params"]), w["q"], w["dt"],
                               w["n_steps"], cot, u0)
    np.testing.assert_allclose(dth, odth, rtol=1e-10, atol=1e-12)
    assert np.abs(du - odu).max() <= 1e-12


def test_adjoint_fp32_vs_oracle(fk, oracle):
    w = dict(SMALL, n_steps=60)
    shape = (w["n"][1], w["n"][0])
    cot = np.random.default_rng(2).standard_normal(shape)
    dth, du = _gpu_adjoint(fk, w, "fp32", cot)
    g = oracle.Grid(w["n"], w["lo"], w["hi"])
    odth, odu = oracle.adjoint(g, oracle.CELLULAR_FLOW, list(w["params"]), w["q"], w["dt"],
                               w["n_steps"], cot)
    rel = np.abs(dth - odth) / np.abs(odth)
    print(f"FP32 adjoint vs FP64 oracle adjoint: relative errors {rel}")
    assert rel.max() <= 1e-3
    assert np.abs(du - odu).max() <= 1e-3 * np.abs(odu).max()


# 41 x 21 mesh, 6 x 6 points, reach about three cells: a 7 x 7 window for
# the masked form, and exits along x, y and both at most nodes
EXITS = dict(n=(41, 21), lo=(0.0, 0.0), hi=(2.0, 1.0), family="cellular_flow",
             params=(1.0, 0.2, 2 * math.pi, 0.05), q=6, dt=1e-2, n_steps=20)


@pytest.mark.parametrize("kernel", ["masked", "scatter"])
def test_adjoint_fp32_forms_vs_oracle(fk, oracle, monkeypatch, kernel):
    """Both FP32 backward forms (masked tensor window, per-point transposed
    scatter) against the FP64 oracle adjoint, from a random terminal field."""
    monkeypatch.setenv("FK_ADJ_KERNEL", kernel)
    w = EXITS
    shape = (w["n"][1], w["n"][0])
    cot = np.random.default_rng(6).standard_normal(shape)
    u0 = fk_inputs.random_field(shape, seed=7)
    dth, du = _gpu_adjoint(fk, w, "fp32", cot, u0, K=7, kernel=kernel)
    g = oracle.Grid(w["n"], w["lo"], w["hi"])
    odth, odu = oracle.adjoint(g, oracle.CELLULAR_FLOW, list(w["params"]), w["q"], w["dt"],
                               w["n_steps"], cot, u0)
    rel = np.abs(dth - odth) / np.abs(odth)
    print(f"{kernel}: FP32 adjoint vs FP64 oracle, parameters rel {rel}, "
          f"terminal field max-abs {np.abs(du - odu).max():.2e} (scale {np.abs(odu).max():.2e})")
    assert rel.max() <= 1e-3
    assert np.abs(du - odu).max() <= 1e-4 * np.abs(odu).max()


@pytest.mark.parametrize("n,q,D", [((5, 3), 4, 0.01), ((9, 5), 4, 0.02), ((33, 17), 4, 0.02)])
def test_adjoint_masked_small_meshes_vs_oracle(fk, oracle, monkeypatch, n, q, D):
    """The masked form on meshes of one tile and of a few: every node is a
    boundary node or next to one, so each tile's kernel forms lambda at its
    nodes and also zeroes the accumulators of the boundary nodes next to
    them, for the step after (three steps' buffers in turn, K = 2)."""
    monkeypatch.setenv("FK_ADJ_KERNEL", "masked")
    w = dict(SMALL, n=n, q=q, n_steps=7, dt=1e-2, params=(1.0, 0.2, 2 * math.pi, D))
    shape = (n[1], n[0])
    cot = np.random.default_rng(8).standard_normal(shape)
    u0 = fk_inputs.random_field(shape, seed=9)
    dth, du = _gpu_adjoint(fk, w, "fp32", cot, u0, K=2, kernel="masked")
    g = oracle.Grid(w["n"], w["lo"], w["hi"])
    odth, odu = oracle.adjoint(g, oracle.CELLULAR_FLOW, list(w["params"]), w["q"], w["dt"],
                               w["n_steps"], cot, u0)
    scale = np.abs(odth).max()
    assert np.abs(dth - odth).max() <= 1e-3 * scale
    assert np.abs(du - odu).max() <= 1e-4 * np.abs(odu).max()


def test_adjoint_checkpoint_interval(fk):
    w = dict(SMALL, n_steps=23)
    shape = (w["n"][1], w["n"][0])
    cot = np.random.default_rng(4).standard_normal(shape)
    res = [_gpu_adjoint(fk, w, "fp64", cot, K=k) for k in (1, 5, 23, 50)]
    for dth, du in res[1:]:
        np.testing.assert_allclose(dth, res[0][0], rtol=1e-12, atol=1e-14)
        assert np.abs(du - res[0][1]).max() <= 1e-14


def _mean_cotangent(shape):
    g = np.zeros(shape)
    g[1:-1, 1:-1] = 1.0 / ((shape[0] - 2) * (shape[1] - 2))
    return g


def test_adjoint_full_size_vs_fd_and_fp64(fk):
    """The adjoint workload: gradients of the mean exit probability at T = 2
    on 1025 x 513 w.r.t. (A, eps, D), checkpoint every 50 steps."""
    import torch
    w = fk_inputs.workload("adjoint_1025x513")
    shape = (w["n"][1], w["n"][0])
    cot = _mean_cotangent(shape)
    d32, du32 = _gpu_adjoint(fk, w, "fp32", cot, K=50)
    d64, du64 = _gpu_adjoint(fk, w, "fp64", cot, K=50)
    g = torch.tensor(cot, device="cuda")

    def L(params):
        p = fk.Plan(_spec(fk, dict(w, params=params), "fp64"))
        v = float((p.solve() * g).sum().item())
        p.close()
        return v

    P = list(w["params"])
    fd = {}
    for k, h in ((0, 1e-4), (1, 1e-4), (3, 1e-4 * P[3])):
        pp, pm = list(P), list(P)
        pp[k] += h
        pm[k] -= h
        fd[k] = (L(pp) - L(pm)) / (2 * h)
    for k in (0, 1, 3):
        rel_fd = abs(d64[k] - fd[k]) / abs(fd[k])
        rel_32 = abs(d32[k] - d64[k]) / abs(d64[k])
        print(f"theta[{k}]: adjoint64 {d64[k]:.9e} fd {fd[k]:.9e} rel {rel_fd:.2e}; "
              f"fp32 vs fp64 rel {rel_32:.2e}")
        assert rel_fd <= 1e-4
        assert rel_32 <= 1e-3


def test_adjoint_full_size_terminal_field(fk):
    """dL/du^N at full size from a random smooth terminal field (from chi the
    interior is flat, where the slope rule has no derivative): FP32 against
    FP64 in relative L2 norm, FP64 against central differences (h = 1e-6)."""
    import torch
    w = fk_inputs.workload("adjoint_1025x513")
    shape = (w["n"][1], w["n"][0])
    cot = _mean_cotangent(shape)
    u0 = fk_inputs.random_field(shape, seed=12)
    d32, du32 = _gpu_adjoint(fk, w, "fp32", cot, u0, K=50)
    d64, du64 = _gpu_adjoint(fk, w, "fp64", cot, u0, K=50)
    rel = np.linalg.norm(du32 - du64) / np.linalg.norm(du64)
    print(f"terminal-field gradient, FP32 vs FP64: relative L2 {rel:.2e}; "
          f"parameters {np.abs(d32 - d64) / np.abs(d64)}")
    # measured 1.7e-3: through 2000 FP32 steps the slope rule's branch
    # weights near its kinks follow the FP32 field
    assert rel <= 5e-3
    assert np.all(np.abs(d32 - d64) <= 1e-3 * np.abs(d64))
    g = torch.tensor(cot, device="cuda")
    plan = fk.Plan(_spec(fk, w, "fp64"))
    base = torch.tensor(u0, device="cuda")
    for idx in ((256, 512), (3, 700), (500, 1)):
        up, um = base.clone(), base.clone()
        up[idx] += 1e-6
        um[idx] -= 1e-6
        fd = float(((plan.solve(up) - plan.solve(um)) * g).sum().item()) / 2e-6
        print(f"du^N{idx}: adjoint {du64[idx]:.6e} fd {fd:.6e}")
        assert abs(du64[idx] - fd) <= 1e-6 * abs(fd) + 1e-12
    plan.close()


def test_autograd_function(fk):
    import torch
    w = dict(SMALL)
    spec = _spec(fk, w, "fp64")
    theta = torch.tensor(w["params"], dtype=torch.float64, requires_grad=True)
    shape = (w["n"][1], w["n"][0])
    ut = torch.tensor(fk_inputs.random_field(shape, seed=8), device="cuda", requires_grad=True)
    u0 = fk.exit_probability(spec, theta, ut, checkpoint_every=4)
    loss = u0[1:-1, 1:-1].mean()
    loss.backward()
    plan = fk.Plan(spec)
    cot = torch.zeros(shape, dtype=torch.float64, device="cuda")
    cot[1:-1, 1:-1] = 1.0 / ((shape[0] - 2) * (shape[1] - 2))
    dth, du = plan.adjoint(cot, ut.detach(), checkpoint_every=4)
    torch.cuda.synchronize()
    plan.close()
    assert torch.allclose(theta.grad, dth.cpu(), rtol=1e-12, atol=1e-15)
    assert torch.allclose(ut.grad, du, rtol=1e-12, atol=1e-15)
