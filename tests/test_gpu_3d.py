"""d = 3 on the GPU (the tensor extension of Sec. 3.1.3), through the C ABI,
against the FP64 oracle on the same seeded inputs.

Tolerances (max-abs): 1e-12 FP64, 1e-5 FP32.  Meshes are ragged (no extent
is a multiple of the 32- to 128-node x-blocks) and small enough for whole
marches; the window width W runs over 3..8 by the choice of dt.  The
129^3 benchmark workload is checked over one step at sampled nodes (the
corners, faces and a centre line included) from a random field, and its
whole FP32 march against the FP64 oracle at a coarser mesh of the same
problem is left to the product-form pin of the oracle.
"""
import math
import os

import numpy as np
import pytest

import fk_inputs

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1
DRIFT = (0.3, -0.2, 0.1, 0.5)


@pytest.fixture(scope="module")
def fk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_14561_gb300 as fk
    fk.load()
    return fk


def _w(n, precision="fp64", params=DRIFT, q=4, dt=2e-3, n_steps=15,
       lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0)):
    return dict(n=n, lo=lo, hi=hi, family="const_drift", params=params, q=q, dt=dt,
                n_steps=n_steps, precision=precision)


def _spec(fk, w, n_steps=None):
    return fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"], params=w["params"],
                       q=w["q"], dt=w["dt"], n_steps=n_steps or w["n_steps"],
                       precision=w["precision"])


def _grid(oracle, w):
    return oracle.Grid(tuple(w["n"]), tuple(w["lo"]), tuple(w["hi"]))


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


def _oracle(oracle, w, k=None, u0=None):
    return oracle.march(_grid(oracle, w), oracle.CONST_DRIFT, list(w["params"]), w["q"], w["dt"],
                        k or w["n_steps"], 0, u0, nthreads=NCPU)


@pytest.mark.parametrize("n", [(37, 21, 19), (45, 33, 9)])
def test_3d_fp64_vs_oracle(fk, oracle, n):
    w = _w(n)
    got, info = _solve(fk, w)
    assert info["step_kernel"] == "window3d" and info["dim"] == 3
    assert got.shape == tuple(reversed(n))
    assert np.abs(got - _oracle(oracle, w)).max() <= 1e-12
    assert got[1:-1, 1:-1, 1:-1].max() > 0.05  # the march moved away from chi


def test_3d_fp32_random_field(fk, oracle):
    w = _w((41, 29, 23), precision="fp32", q=6, n_steps=12)
    u0 = fk_inputs.random_field((23, 29, 41), seed=61)
    got, _ = _solve(fk, w, u0)
    assert np.abs(got - _oracle(oracle, w, u0=u0)).max() <= 1e-5


@pytest.mark.parametrize("dt,W", [(2e-4, 3), (1.5e-3, 4), (4.5e-3, 5), (9e-3, 6), (1.4e-2, 7),
                                  (2.2e-2, 8)])
def test_3d_window_widths(fk, oracle, dt, W):
    """One step from a random field for every window width the kernel is
    built for (the point spread grows with dt), FP64."""
    import torch
    w = _w((33, 25, 27), dt=dt, n_steps=3, q=4, params=(0.9, -0.7, 0.4, 0.5))
    plan = fk.Plan(_spec(fk, w))
    assert plan.info()["window_rows"] == W
    u1 = fk_inputs.random_field((27, 25, 33), seed=62 + W)
    got = plan.march(2, 1, torch.tensor(u1, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    plan.close()
    want = oracle.march(_grid(oracle, w), oracle.CONST_DRIFT, list(w["params"]), 4, dt, 2, 1, u1)
    assert np.abs(got.cpu().numpy() - want).max() <= 1e-12


def test_3d_too_wide_rejected(fk):
    with pytest.raises(fk.FkError):
        fk.Plan(_spec(fk, _w((33, 25, 27), dt=4e-2, params=(0.9, -0.7, 0.4, 0.5))))


def test_3d_horizons_and_snapshots(fk, oracle):
    import torch
    w = _w((29, 23, 21), n_steps=6)
    plan = fk.Plan(_spec(fk, w))
    hz = plan.solve_horizons()
    snaps = torch.empty((3,) + plan.shape, dtype=torch.float64, device="cuda")
    u0 = plan.solve(snapshots=snaps, snapshot_stride=2)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    hz, snaps, u0 = hz.cpu().numpy(), snaps.cpu().numpy(), u0.cpu().numpy()
    plan.close()
    for k in (1, 4, 6):
        assert np.abs(hz[k - 1] - _oracle(oracle, w, k)).max() <= 1e-12, k
    assert np.array_equal(snaps[-1], u0)
    assert np.array_equal(hz[-1], u0)


def test_3d_workload_sampled_step(fk, oracle):
    """The 129^3 benchmark workload (FP32, 4^3 points): one step from a random
    field at sampled nodes against the oracle's step there; the whole march
    stays in [0, 1]."""
    import torch
    w = fk_inputs.workload("drift3d_129")
    shape = tuple(reversed(w["n"]))
    plan = fk.Plan(_spec(fk, w))
    assert plan.info()["window_rows"] == 7
    u1 = fk_inputs.random_field(shape, seed=63)
    n = 250
    got = plan.march(n + 1, n, torch.tensor(u1, dtype=torch.float32, device="cuda"))
    got = got.double().cpu().numpy().reshape(-1)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    nodes = fk_inputs.sample_nodes(shape, 3000, seed=9)
    want = oracle.step_nodes(_grid(oracle, w), oracle.CONST_DRIFT, list(w["params"]), w["q"],
                             w["dt"], n, u1, nodes, nthreads=NCPU)
    assert np.abs(got[nodes] - want).max() <= 1e-5
    full = plan.solve().double().cpu().numpy()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    plan.close()
    assert full.min() >= -1e-6 and full.max() <= 1 + 1e-6
    # the centre is ~3 standard deviations from every face: 1 - prod of the
    # 1D survivals there is 0.037
    assert 0.02 < full[64, 64, 64] < 0.06


def test_3d_full_march_vs_product_form(fk, oracle):
    """The whole 500-step FP32 march of the benchmark workload against the
    continuous answer 1 - prod_m S_m (independent components; S_m the 1D
    survival in closed form): the scheme's own error on this mesh, pinned
    on the oracle at coarser meshes, stays below 1e-2 in rms."""
    import torch
    w = fk_inputs.workload("drift3d_129")
    plan = fk.Plan(_spec(fk, w))
    u = plan.solve().double().cpu().numpy()
    torch.cuda.synchronize()
    plan.close()
    T = w["dt"] * w["n_steps"]
    g = _grid(oracle, w)
    s = [1 - oracle.exit_prob_1d_image(g.axis(m), T, -1, 1, w["params"][m], w["params"][3])
         for m in range(3)]
    ref = 1 - np.einsum("k,j,i->kji", s[2], s[1], s[0])
    rms = math.sqrt(np.mean((u - ref) ** 2))
    print(f"drift3d_129 fp32 vs product form: rms {rms:.3e}, max {np.abs(u - ref).max():.3e}")
    assert rms < 1e-2
