"""Algorithm 1 (Sec. 3.2) on the GPU: fk_solve_horizons gives P(t_k, .) for
every horizon k = 1..N in one pass, through the C ABI.

Horizon k is the march of Scheme 1 over k steps with the coefficients of
t_{k-1}, ..., t_0, so each output field is checked against
* the FP64 oracle's march of k steps (1e-12 FP64, 1e-5 FP32, max-abs);
* the library's own single-field march with n_steps = k, which runs the
  same kernel on the same tile: the fields must agree bit for bit (a
  row-window plan advances several fields with the direct kernel, so there
  to FP32 rounding);
and the whole set against the property that P(t_k) does not decrease in k
(to rounding on a resolved grid, as the oracle pins).
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


def _spec(fk, w, n_steps=None):
    return fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"],
                       params=w["params"], q=w["q"], dt=w["dt"],
                       n_steps=n_steps or w["n_steps"], precision=w["precision"],
                       path=w.get("path", "matrix_free"))


def _horizons(fk, w, u_terminal=None):
    import torch
    plan = fk.Plan(_spec(fk, w))
    ut = None if u_terminal is None else torch.tensor(u_terminal, dtype=plan.dtype, device="cuda")
    out = plan.solve_horizons(ut)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    info = plan.info()
    res = out.cpu().numpy()
    plan.close()
    return res, info


def _single(fk, w, k, u_terminal=None):
    import torch
    plan = fk.Plan(_spec(fk, w, n_steps=k))
    ut = None if u_terminal is None else torch.tensor(u_terminal, dtype=plan.dtype, device="cuda")
    out = plan.solve(ut)
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    plan.close()
    return res


def _oracle(oracle, w, k, u_terminal=None):
    g = oracle.Grid(tuple(w["n"]), tuple(w["lo"]), tuple(w["hi"]))
    fam = {"const_drift": oracle.CONST_DRIFT, "cellular_flow": oracle.CELLULAR_FLOW}[w["family"]]
    return oracle.march(g, fam, list(w["params"]), w["q"], w["dt"], k, 0, u_terminal,
                        nthreads=NCPU)


def _w2d(n, q, precision, n_steps, dt=2e-3, D=5e-3, eps=0.3):
    return fk_inputs.workload("cellular_1025x513", n=n, q=q, n_steps=n_steps, dt=dt,
                              precision=precision, params=(1.0, eps, 2 * math.pi, D))


def test_horizons_fp64_vs_oracle_and_single(fk, oracle):
    w = _w2d((77, 41), 4, "fp64", 12)
    got, _ = _horizons(fk, w)
    assert got.shape == (12, 41, 77)
    for k in range(1, 13):
        assert np.abs(got[k - 1] - _oracle(oracle, w, k)).max() <= 1e-12, k
    for k in (1, 5, 12):
        assert np.array_equal(got[k - 1], _single(fk, w, k)), k


@pytest.mark.parametrize("kernel", ["direct", "window", "masked"])
def test_horizons_fp32_kernels(fk, oracle, monkeypatch, kernel):
    """The FP32 plans of each step kernel.  The direct and masked kernels
    take the fields through their grid's z index and match the single march
    bit for bit; a row-window plan advances several fields with the direct
    kernel on every row, equal to its single march up to FP32 rounding."""
    monkeypatch.setenv("FK_STEP_KERNEL", kernel)
    w = _w2d((161, 81), 6, "fp32", 10, dt=1e-3, D=0.025)
    got, info = _horizons(fk, w)
    assert info["step_kernel"] == kernel
    for k in (1, 2, 7, 10):
        single = _single(fk, w, k)
        if kernel == "window":
            assert np.abs(got[k - 1] - single).max() <= 1e-6, k
        else:
            assert np.array_equal(got[k - 1], single), k
        assert np.abs(got[k - 1] - _oracle(oracle, w, k)).max() <= 1e-5, k


def test_horizons_terminal_field(fk, oracle):
    w = _w2d((53, 29), 6, "fp64", 8)
    u0 = fk_inputs.random_field((29, 53), seed=21)
    got, _ = _horizons(fk, w, u0)
    for k in (1, 4, 8):
        assert np.abs(got[k - 1] - _oracle(oracle, w, k, u0)).max() <= 1e-12, k


def test_horizons_1d(fk, oracle):
    w = fk_inputs.workload("bm1d_drift", n=(61,), n_steps=9)
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        w = dict(w, precision=prec)
        got, _ = _horizons(fk, w)
        assert got.shape == (9, 61)
        for k in (1, 3, 9):
            assert np.abs(got[k - 1] - _oracle(oracle, w, k)).max() <= tol, (prec, k)


def test_horizons_monotone_in_k(fk):
    """The resolved case of the oracle pin: 129 x 65, dt = 5e-3, 30 horizons."""
    w = _w2d((129, 65), 4, "fp64", 30, dt=5e-3, D=2e-3)
    got, _ = _horizons(fk, w)
    worst = float(np.diff(got, axis=0).min())
    print(f"horizons 129x65: worst decrease in k {worst:.2e}")
    assert worst >= -1e-13
    assert got[-1, 1:-1, 1:-1].max() > 0.05


def test_horizons_full_size_columns(fk):
    """The 200-horizon benchmark workload on 1025 x 513 (FP32, masked kernel):
    fields 1, 100 and 200 equal the single marches of 1, 100 and 200 steps
    bit for bit (the single march is checked against the oracle at this size
    by the march tests)."""
    w = fk_inputs.workload("horizons_1025x513")
    got, info = _horizons(fk, w)
    assert info["step_kernel"] == "masked"
    for k in (1, 100, 200):
        assert np.array_equal(got[k - 1], _single(fk, w, k)), k


def test_horizons_errors(fk):
    import torch
    w = _w2d((33, 17), 4, "fp64", 5)
    plan = fk.Plan(_spec(fk, w))
    out = torch.empty((5, 17, 33), dtype=torch.float64, device="cuda")
    with pytest.raises(fk.FkError):  # terminal field inside the output
        plan.solve_horizons(out[2], out)
    plan.close()
    wc = dict(_w2d((33, 17), 4, "fp64", 5, eps=0.0), path="csr")
    plan = fk.Plan(_spec(fk, wc))
    with pytest.raises(fk.FkError):
        plan.solve_horizons()
    plan.close()
