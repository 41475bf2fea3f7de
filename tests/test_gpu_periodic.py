"""Periodic x and the paper's own 2D example (Sec. 4.2) on the GPU, through
the C ABI, against the FP64 oracle on the same seeded inputs.

Tolerances (max-abs): 1e-12 FP64, 1e-5 FP32.  Meshes have ragged last tiles
in x (the period is not a multiple of the 32-column tile) and are small
enough for whole-march parity; the benchmark's 1025 x 257 workload is checked
over one step at sampled nodes from a random periodic field, and its column
0 against column nx - 1.
"""
import math
import os

import numpy as np
import pytest

import fk_inputs

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1
PAPER = (10.0, 2.0, 0.15, 2 * math.pi / 10)


@pytest.fixture(scope="module")
def fk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_14561_gb300 as fk
    fk.load()
    return fk


def _w(n, precision="fp64", family="paper_cellular", params=PAPER, q=4, dt=2e-4, n_steps=20,
       lo=(-math.pi, 0.0), hi=(math.pi, 1.0)):
    return dict(n=n, lo=lo, hi=hi, family=family, params=params, q=q, dt=dt, n_steps=n_steps,
                precision=precision, periodic_x=True, path="matrix_free")


def _spec(fk, w, n_steps=None):
    return fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"], params=w["params"],
                       q=w["q"], dt=w["dt"], n_steps=n_steps or w["n_steps"],
                       precision=w["precision"], periodic_x=True)


def _oracle_grid(oracle, w):
    return oracle.Grid(tuple(w["n"]), tuple(w["lo"]), tuple(w["hi"]), periodic=1)


def _periodic_field(shape, seed):
    u = fk_inputs.random_field(shape, seed=seed, boundary_one=False)
    u[0, :] = 1.0
    u[-1, :] = 1.0
    u[:, -1] = u[:, 0]
    return u


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


@pytest.mark.parametrize("n", [(45, 21), (129, 65), (70, 40)])
def test_paper_fp64_vs_oracle(fk, oracle, n):
    w = _w(n)
    got, info = _solve(fk, w)
    assert info["step_kernel"] == "direct" and info["periodic_x"] and not info["nonuniform"]
    want = oracle.march(_oracle_grid(oracle, w), oracle.PAPER_CELLULAR, list(PAPER), w["q"],
                        w["dt"], w["n_steps"], 0, nthreads=NCPU)
    assert np.abs(got - want).max() <= 1e-12
    assert np.array_equal(got[:, 0], got[:, -1])
    assert got[1:-1, 1:-1].max() > 0.05  # the march moved away from chi


def test_paper_fp32_vs_oracle_random_field(fk, oracle):
    w = _w((97, 49), precision="fp32", q=6, n_steps=30)
    u0 = _periodic_field((49, 97), seed=41)
    got, _ = _solve(fk, w, u0)
    want = oracle.march(_oracle_grid(oracle, w), oracle.PAPER_CELLULAR, list(PAPER), 6, w["dt"],
                        w["n_steps"], 0, u0, nthreads=NCPU)
    assert np.abs(got - want).max() <= 1e-5
    assert np.array_equal(got[:, 0], got[:, -1])


def test_const_drift_periodic_vs_oracle(fk, oracle):
    """A drift across the seam (b_1 = 0.9): every shifted point near x = lo
    or x = hi wraps to the other side."""
    w = _w((61, 33), family="const_drift", params=(0.9, -0.3, 0.0, 0.6), lo=(0.0, -1.0),
           hi=(2.0, 1.0), dt=2e-3, n_steps=25)
    u0 = _periodic_field((33, 61), seed=43)
    got, _ = _solve(fk, w, u0)
    want = oracle.march(_oracle_grid(oracle, w), oracle.CONST_DRIFT, list(w["params"]), w["q"],
                        w["dt"], w["n_steps"], 0, u0, nthreads=NCPU)
    assert np.abs(got - want).max() <= 1e-12


def test_periodic_horizons(fk, oracle):
    import torch
    w = _w((53, 29), n_steps=8)
    plan = fk.Plan(_spec(fk, w))
    out = plan.solve_horizons()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    plan.close()
    for k in (1, 4, 8):
        want = oracle.march(_oracle_grid(oracle, w), oracle.PAPER_CELLULAR, list(PAPER), w["q"],
                            w["dt"], k, 0, nthreads=NCPU)
        assert np.abs(got[k - 1] - want).max() <= 1e-12, k


def test_periodic_batched_equals_single(fk):
    import torch
    ws = [_w((45, 21), precision="fp32"), _w((77, 37), precision="fp32", q=4)]
    singles = [_solve(fk, w)[0] for w in ws]
    plans = [fk.Plan(_spec(fk, w)) for w in ws]
    outs = fk.solve_batched(plans)
    torch.cuda.synchronize()
    for o, s in zip(outs, singles):
        assert np.array_equal(o.double().cpu().numpy(), s)
    for p in plans:
        p.close()


def test_periodic_adjoint_unsupported(fk):
    import torch
    plan = fk.Plan(_spec(fk, _w((45, 21))))
    with pytest.raises(fk.FkError):
        plan.adjoint(torch.zeros(plan.shape, dtype=torch.float64, device="cuda"))
    plan.close()


def test_paper_workload_sampled_step(fk, oracle):
    """The benchmark workload (1025 x 257, 6 x 6 points, FP32): one step from
    a random periodic field at 2000 sampled nodes (every boundary-adjacent
    row and the seam columns included) against the oracle's step at those
    nodes; the full march keeps columns 0 and nx-1 equal."""
    import torch
    w = fk_inputs.workload("paper_2d_1025x257")
    ny, nx = w["n"][1], w["n"][0]
    u1 = _periodic_field((ny, nx), seed=47)
    plan = fk.Plan(_spec(fk, w, n_steps=w["n_steps"]))
    ut = torch.tensor(u1, dtype=torch.float32, device="cuda")
    n = 377
    got = plan.march(n + 1, n, ut).double().cpu().numpy()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    nodes = fk_inputs.sample_nodes((ny, nx), 2000, seed=5)
    seam = np.concatenate([np.arange(ny) * nx, np.arange(ny) * nx + nx - 1,
                           np.arange(ny) * nx + 1, np.arange(ny) * nx + nx - 2])
    nodes = np.unique(np.concatenate([nodes, seam]))
    want = oracle.step_nodes(_oracle_grid(oracle, w), oracle.PAPER_CELLULAR, list(PAPER), w["q"],
                             w["dt"], n, u1, nodes, nthreads=NCPU)
    assert np.abs(got.reshape(-1)[nodes] - want).max() <= 1e-5
    full = plan.solve().cpu().numpy()
    assert np.array_equal(full[:, 0], full[:, -1])
    assert full[1:-1, 1:-1].max() > 0.05
    plan.close()


def test_paper_workload_full_march_vs_golden(fk):
    """The paper's example at the benchmark's size: all 1000 FP32 steps
    against the FP64 oracle's u^0 at 22k sampled nodes (the rows next to the
    y faces and the seam columns included), written by
    tests/golden/make_oracle_golden.py."""
    import torch
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden",
                                "paper_2d_1025x257_oracle_u0.npz"))
    w = fk_inputs.workload("paper_2d_1025x257")
    assert tuple(gold["n"]) == tuple(w["n"]) and int(gold["n_steps"]) == w["n_steps"]
    plan = fk.Plan(_spec(fk, w))
    out = plan.solve()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    got = out.double().reshape(-1).cpu().numpy()[gold["nodes"]]
    plan.close()
    err = np.abs(got - gold["u0"]).max()
    print(f"paper_2d_1025x257 fp32 vs fp64 oracle, 1000 steps: max-abs {err:.3e}")
    assert err <= 1e-5
