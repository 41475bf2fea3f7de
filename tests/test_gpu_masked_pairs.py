"""GPU parity of the masked tensor-window kernel with two nodes per thread
(register variant 3: nodes (i, k) and (i, k + 1) read the rows their
windows share once), through the C ABI, against the FP64 oracle.

The variant is forced with FK_STEP_TILE=<even height>,3,2, so every case
runs it whatever the plan's timing would pick:
* the window width it is built for, W = 7, on meshes from 17 x 9 to
  161 x 81, 100 steps, max-abs 1e-5 against the oracle (plans of other
  widths refuse it and keep one node per thread); ragged last tiles leave a lone last row (its partner is the
  boundary row, computed but not stored);
* steps of 1e-2 and 2e-2 with strong flows, where floor(drift) steps
  between neighbouring rows, so that B's window starts 0, 1 or 2 rows below
  A's and one column to either side (and, at the strongest flow, further:
  the pair then takes the two windows one after the other);
* the persistent march of the variant, bit for bit against its per-step
  launches, and Algorithm 1's fields against single marches bit for bit;
* the 2000-step benchmark march against the oracle's golden values.
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


@pytest.fixture
def pairs(monkeypatch):
    """Plans created in the test run the masked kernel's variant 3."""
    monkeypatch.setenv("FK_STEP_KERNEL", "masked")
    monkeypatch.setenv("FK_STEP_TILE", "16,3,2")
    monkeypatch.setenv("FK_MARCH", "steps")
    return monkeypatch


def _spec(fk, w, n_steps=None):
    return fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"],
                       params=w["params"], q=w["q"], dt=w["dt"],
                       n_steps=n_steps or w["n_steps"], precision="fp32")


def _cellular(n, q, D, dt, n_steps, A=1.0):
    return fk_inputs.workload("cellular_1025x513", n=n, q=q, n_steps=n_steps, precision="fp32",
                              params=(A, 0.2, 2 * math.pi, D), dt=dt)


def _oracle(oracle, w, n_from, n_to=0, u_in=None):
    g = oracle.Grid(tuple(w["n"]), tuple(w["lo"]), tuple(w["hi"]))
    return oracle.march(g, FAM[w["family"]], list(w["params"]), w["q"], w["dt"], n_from, n_to,
                        u_in, nthreads=NCPU)


def _solve(fk, w, u0=None, n_steps=None):
    import torch
    plan = fk.Plan(_spec(fk, w, n_steps))
    info = plan.info()
    ut = None if u0 is None else torch.tensor(u0, dtype=torch.float32, device="cuda")
    out = plan.solve(ut)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    res = out.double().cpu().numpy()
    plan.close()
    return res, info


# (mesh, Q, D, dt, A, W): isotropic meshes on [0,2]x[0,1]
PAIR_CASES = [
    ((161, 81), 6, 0.035, 1e-3, 1.0, 7),
    ((161, 81), 4, 0.07, 1e-3, 1.0, 7),
    ((41, 21), 6, 0.05, 1e-2, 1.0, 7),
    ((81, 41), 6, 0.015, 1e-2, 2.0, 7),
    ((17, 9), 6, 0.35, 1e-2, 1.0, 7),
    ((41, 21), 4, 0.055, 2e-2, 10.0, 7),
]


@pytest.mark.parametrize("n,q,D,dt,A,W", PAIR_CASES)
def test_pairs_vs_oracle(fk, oracle, pairs, n, q, D, dt, A, W):
    w = _cellular(n, q, D, dt, 100, A=A)
    got, info = _solve(fk, w)
    assert info["step_kernel"] == "masked" and info["window_rows"] == W
    assert info["nodes_per_thread"] == 2 and info["tile"][1] == 16
    err = np.abs(got - _oracle(oracle, w, w["n_steps"])).max()
    assert err <= TOL32, err


@pytest.mark.parametrize("seed", [3, 4])
def test_pairs_random_field(fk, oracle, pairs, seed):
    """From a random terminal field (slopes of both signs at every face and
    corner), 5 steps on a 101 x 51 mesh with 10-row tiles (odd tile rows:
    the last tile's lone row)."""
    pairs.setenv("FK_STEP_TILE", "10,3,2")
    w = _cellular((101, 51), 6, 0.045, 2e-3, 5)
    u0 = fk_inputs.random_field((51, 101), seed=seed)
    got, info = _solve(fk, w, u0)
    assert info["nodes_per_thread"] == 2 and info["window_rows"] == 7
    assert np.abs(got - _oracle(oracle, w, 5, 0, u0)).max() <= TOL32


@pytest.mark.parametrize("q,D,W", [(8, 0.05, 9), (4, 0.03, 5)])
def test_pairs_refused_for_other_widths(fk, pairs, q, D, W):
    """Plans of other window widths asked for variant 3 keep one node per
    thread."""
    w = _cellular((161, 81), q, D, 1e-3, 5)
    _, info = _solve(fk, w)
    assert info["step_kernel"] == "masked" and info["window_rows"] == W
    assert info["nodes_per_thread"] == 1


def test_pairs_persistent_march_bit_for_bit(fk, oracle, pairs):
    """The persistent march of variant 3 equals its per-step launches bit
    for bit, and the oracle to 1e-5."""
    w = _cellular((161, 81), 6, 0.035, 1e-3, 101)
    res = {}
    for mode in ("persistent", "steps"):
        pairs.setenv("FK_MARCH", mode)
        res[mode], info = _solve(fk, w)
        assert info["march_mode"] == mode and info["nodes_per_thread"] == 2
    assert np.array_equal(res["persistent"], res["steps"])
    assert np.abs(res["steps"] - _oracle(oracle, w, 101)).max() <= TOL32


def test_pairs_horizons_equal_single_marches(fk, oracle, pairs):
    """Algorithm 1's fields (several per launch) run the same paired tile
    code as a single march: bit for bit."""
    import torch
    w = _cellular((161, 81), 4, 0.07, 1e-3, 10)
    plan = fk.Plan(_spec(fk, w))
    assert plan.info()["nodes_per_thread"] == 2
    got = plan.solve_horizons()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    got = got.cpu().numpy()
    plan.close()
    for k in (1, 4, 10):
        single, info = _solve(fk, w, n_steps=k)
        assert info["nodes_per_thread"] == 2
        assert np.array_equal(got[k - 1], single.astype(np.float32)), k
        assert np.abs(got[k - 1] - _oracle(oracle, w, k)).max() <= TOL32, k


def test_pairs_benchmark_march_vs_golden(fk, pairs):
    """The 2000-step 1025 x 513 march with variant 3 (58-row tiles: 288 tiles,
    all resident at 2 per SM, so the persistent march applies) against
    the FP64 oracle's u^0 at the golden nodes."""
    import torch
    pairs.setenv("FK_STEP_TILE", "58,3,2")
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden",
                                "cellular_1025x513_oracle_u0.npz"))
    w = fk_inputs.workload("cellular_1025x513")
    for mode in ("steps", "persistent"):
        pairs.setenv("FK_MARCH", mode)
        plan = fk.Plan(_spec(fk, w))
        info = plan.info()
        assert info["nodes_per_thread"] == 2 and info["march_mode"] == mode
        out = plan.solve()
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        got = out.double().reshape(-1).cpu().numpy()[gold["nodes"]]
        plan.close()
        assert np.abs(got - gold["u0"]).max() <= TOL32, mode
