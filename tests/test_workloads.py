"""The benchmark's workloads on CPU: each is the configuration its name and
the measured metric stand for, so that a change to a size, a rule or a step
count cannot pass unnoticed into the timed runs."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import fk_inputs  # noqa: E402


def test_headline_workload_is_the_cellular_flow_march():
    """1025 x 513 nodes on [0, 2] x [0, 1], psi = A sin(pi x) sin(pi y) +
    eps sin(omega t) sin(2 pi x) sin(pi y) with A = 1, eps = 0.2, omega =
    2 pi, D = 1e-3; 6 x 6 points, dt = 1e-3, 2000 steps, FP32."""
    w = fk_inputs.workload("cellular_1025x513")
    assert w["n"] == (1025, 513) and w["lo"] == (0.0, 0.0) and w["hi"] == (2.0, 1.0)
    assert w["family"] == "cellular_flow"
    A, eps, om, D = w["params"]
    assert (A, eps, D) == (1.0, 0.2, 1e-3) and om == pytest.approx(2 * math.pi)
    assert (w["q"], w["dt"], w["n_steps"], w["precision"]) == (6, 1e-3, 2000, "fp32")


def test_the_other_configurations():
    c1 = fk_inputs.workload("bm1d_drift")
    assert c1["n"] == (201,) and c1["lo"] == (-1.0,) and c1["hi"] == (1.0,)
    assert c1["params"][0] == 0.5 and c1["params"][3] == 1.0  # b, sigma
    assert (c1["q"], c1["dt"], c1["n_steps"], c1["precision"]) == (8, 1e-3, 1000, "fp64")
    c3 = fk_inputs.workload("cellular_4097x2049")
    assert c3["n"] == (4097, 2049) and (c3["q"], c3["dt"], c3["n_steps"]) == (8, 5e-4, 4000)
    assert c3["params"] == fk_inputs.workload("cellular_1025x513")["params"]
    c3a = fk_inputs.workload("cellular_autonomous_2049x1025")
    assert c3a["n"] == (2049, 1025) and c3a["path"] == "csr" and c3a["params"][1] == 0.0
    assert (c3a["q"], c3a["dt"], c3a["n_steps"]) == (8, 5e-4, 4000)
    c5 = fk_inputs.workload("adjoint_1025x513")
    head = fk_inputs.workload("cellular_1025x513")
    assert all(c5[k] == head[k] for k in ("n", "lo", "hi", "family", "params", "q", "dt",
                                          "n_steps"))


def test_the_batched_sweep():
    """64 instances, nx odd and uniform in [257, 2049], ny = (nx + 1) / 2,
    D log-uniform in [1e-4, 1e-2], A uniform in [0.5, 2], 6 x 6 points,
    1000 steps, FP32, one fixed seed."""
    ws = fk_inputs.batch("batched_64")
    assert len(ws) == 64
    assert ws == fk_inputs.batch("batched_64")  # seeded
    for w in ws:
        nx, ny = w["n"]
        assert 257 <= nx <= 2049 and nx % 2 == 1 and ny == (nx + 1) // 2
        A, eps, om, D = w["params"]
        assert 0.5 <= A <= 2.0 and 1e-4 <= D <= 1e-2 and eps == 0.2
        assert (w["q"], w["dt"], w["n_steps"], w["precision"]) == (6, 1e-3, 1000, "fp32")
    logD = np.log10([w["params"][3] for w in ws])
    assert logD.min() < -3.5 and logD.max() > -2.5  # spread over the range


def test_units_of_the_metric():
    """Node-quadrature updates per march: interior nodes x Q^d x steps
    (522,753 x 36 x 2000 on the headline workload)."""
    import bench
    w = fk_inputs.workload("cellular_1025x513")
    assert bench.units_per_solve(w) == 1023 * 511 * 36 * 2000
    p = fk_inputs.workload("paper_2d_1025x257")  # periodic x: 1024 distinct columns
    assert bench.units_per_solve(p) == 1024 * 255 * 36 * 1000
    args = _default_args(bench)  # `python bench.py` with no flags: the headline line
    assert args.workload == "cellular_1025x513" and args.gpus == 1 and bench.headline(args)


def _default_args(bench):
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        return bench.parse()
    finally:
        sys.argv = argv
