"""GPU parity of the matrix-free march (libfk_gb300 through the C ABI) with
the FP64 CPU oracle, on the same seeded inputs.

Tolerances (max-abs over every node): 1e-12 for the FP64 path, 1e-5 for
the FP32 path against the FP64 oracle.  Small meshes span several CTA tiles
and a ragged last tile; the full-size workloads are checked over the whole
march where the oracle finishes in tens of seconds, else over a few steps
on the whole mesh and one step on sampled nodes.
"""
import math
import os

import numpy as np
import pytest

import fk_inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5
NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module")
def fk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_14561_gb300 as fk
    fk.load()
    return fk


def _spec(fk, w):
    return fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"],
                       params=w["params"], q=w["q"], dt=w["dt"], n_steps=w["n_steps"],
                       precision=w.get("precision", "fp32"), path=w.get("path", "matrix_free"))


def _oracle_grid(oracle, w):
    return oracle.Grid(tuple(w["n"]), tuple(w["lo"]), tuple(w["hi"]))


FAM = {"const_drift": 0, "cellular_flow": 1}


def _oracle_march(oracle, w, n_from, n_to, u_in=None):
    g = _oracle_grid(oracle, w)
    return oracle.march(g, FAM[w["family"]], list(w["params"]), w["q"], w["dt"], n_from, n_to,
                        u_in, nthreads=NCPU)


def _gpu_solve(fk, w, u_terminal=None):
    import torch
    plan = fk.Plan(_spec(fk, w))
    ut = None if u_terminal is None else torch.tensor(u_terminal, dtype=plan.dtype, device="cuda")
    out = plan.solve(ut)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    res = out.double().cpu().numpy()
    plan.close()
    return res


def _gpu_solve_info(fk, w, u_terminal=None):
    import torch
    plan = fk.Plan(_spec(fk, w))
    info = plan.info()
    ut = None if u_terminal is None else torch.tensor(u_terminal, dtype=plan.dtype, device="cuda")
    out = plan.solve(ut)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    res = out.double().cpu().numpy()
    plan.close()
    return res, info


def _small2d(q, precision, family="cellular_flow", n_steps=20, n=(77, 41)):
    w = fk_inputs.workload("cellular_1025x513", n=n, q=q, n_steps=n_steps,
                           precision=precision, params=(1.0, 0.2, 2 * math.pi, 0.02))
    if family == "const_drift":
        w.update(family="const_drift", params=(0.7, -0.4, 0.0, 0.3))
    return w


def test_gauss_hermite_matches_oracle(fk, oracle):
    for q in range(1, 17):
        a, w = fk.gauss_hermite(q)
        ao, wo = oracle.gauss_hermite(q)
        np.testing.assert_allclose(a, ao, atol=2e-14)
        np.testing.assert_allclose(w, wo, atol=2e-15)


KERNEL1D = {"step": "direct", "resident": "resident", "cluster": "cluster"}


@pytest.fixture(params=["step", "resident", "cluster"])
def kernel1d(request, monkeypatch):
    """1D path of the test's plans: one launch per step, the whole march in
    one CTA, or in one thread-block cluster."""
    monkeypatch.setenv("FK_1D_KERNEL", request.param)
    return request.param


def test_bm1d_drift_fp64_full_march(fk, oracle, kernel1d):
    w = fk_inputs.workload("bm1d_drift")
    got, info = _gpu_solve_info(fk, w)
    assert info["step_kernel"] == KERNEL1D[kernel1d]
    want = _oracle_march(oracle, w, w["n_steps"], 0)
    assert np.abs(got - want).max() <= TOL64


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6, 7, 8])
def test_small2d_fp64_all_q(fk, oracle, q):
    w = _small2d(q, "fp64")
    got = _gpu_solve(fk, w)
    want = _oracle_march(oracle, w, w["n_steps"], 0)
    assert np.abs(got - want).max() <= TOL64


@pytest.mark.parametrize("q", [3, 6, 8])
def test_small2d_fp32(fk, oracle, q):
    w = _small2d(q, "fp32", n_steps=200)
    got = _gpu_solve(fk, w)
    want = _oracle_march(oracle, w, w["n_steps"], 0)
    assert np.abs(got - want).max() <= TOL32


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_small2d_const_drift(fk, oracle, precision, tol):
    w = _small2d(4, precision, family="const_drift", n_steps=60)
    got = _gpu_solve(fk, w)
    want = _oracle_march(oracle, w, w["n_steps"], 0)
    assert np.abs(got - want).max() <= tol


@pytest.mark.parametrize("q", [1, 3, 8, 12, 16])
def test_1d_random_field_fp64(fk, oracle, q, kernel1d):
    w = fk_inputs.workload("bm1d_drift", n=(1500,), q=q, n_steps=7)
    u0 = fk_inputs.random_field((1500,), seed=q)
    got = _gpu_solve(fk, w, u0)
    want = _oracle_march(oracle, w, w["n_steps"], 0, u0)
    assert np.abs(got - want).max() <= TOL64


def test_random_terminal_field_2d(fk, oracle):
    w = _small2d(6, "fp64", n=(101, 67), n_steps=5)
    u0 = fk_inputs.random_field((67, 101), seed=3)
    got = _gpu_solve(fk, w, u0)
    want = _oracle_march(oracle, w, w["n_steps"], 0, u0)
    assert np.abs(got - want).max() <= TOL64


def test_cellular_1025x513_fp32_full_march(fk):
    """The benchmark workload itself: 2000 FP32 steps against the FP64
    oracle's u^0 at 20k+ sampled nodes (all nodes next to the boundary
    included), written by tests/golden/make_oracle_golden.py."""
    import torch
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden",
                                "cellular_1025x513_oracle_u0.npz"))
    w = fk_inputs.workload("cellular_1025x513")
    assert tuple(gold["n"]) == tuple(w["n"]) and int(gold["n_steps"]) == w["n_steps"]
    plan = fk.Plan(_spec(fk, w))
    out = plan.solve()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    got = out.double().reshape(-1).cpu().numpy()[gold["nodes"]]
    plan.close()
    err = np.abs(got - gold["u0"]).max()
    print(f"cellular_1025x513 fp32 vs fp64 oracle, 2000 steps: max-abs {err:.3e}")
    assert err <= TOL32


def test_cellular_1025x513_fp64_60_steps(fk, oracle):
    w = fk_inputs.workload("cellular_1025x513", precision="fp64", n_steps=60)
    got = _gpu_solve(fk, w)
    want = _oracle_march(oracle, w, w["n_steps"], 0)
    assert np.abs(got - want).max() <= TOL64


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("fp32", 2e-6)])
def test_cellular_4097x2049_sampled_step(fk, oracle, precision, tol):
    """One step at full size from a seeded field, checked on sampled nodes."""
    import torch
    w = fk_inputs.workload("cellular_4097x2049", precision=precision)
    shape = (w["n"][1], w["n"][0])
    u1 = fk_inputs.random_field(shape, seed=7)
    plan = fk.Plan(_spec(fk, w))
    n = 1234
    ut = torch.tensor(u1, dtype=plan.dtype, device="cuda")
    out = plan.march(n + 1, n, ut)
    torch.cuda.synchronize()
    nodes = fk_inputs.sample_nodes(shape, 4000, seed=11)
    got = out.double().reshape(-1)[torch.tensor(nodes, device="cuda")].cpu().numpy()
    g = _oracle_grid(oracle, w)
    want = oracle.step_nodes(g, 1, list(w["params"]), w["q"], w["dt"], n, u1, nodes, nthreads=NCPU)
    assert plan.last_device_error() == 0
    plan.close()
    assert np.abs(got - want).max() <= tol


def test_cellular_4097x2049_fp64_two_steps(fk, oracle):
    w = fk_inputs.workload("cellular_4097x2049", precision="fp64", n_steps=2)
    got = _gpu_solve(fk, w)
    want = _oracle_march(oracle, w, 2, 0)
    assert np.abs(got - want).max() <= TOL64


@pytest.mark.parametrize("precision,tol", [("fp32", TOL32), ("fp64", TOL64)])
def test_cellular_4097x2049_50_steps_vs_golden(fk, precision, tol):
    """The large workload's mesh and rule (8 x 8 points, W about 19: the
    direct kernel) over a 50-step march from chi, against the FP64 oracle's
    u^0 at 20k+ sampled nodes (all nodes next to the boundary included),
    written by tests/golden/make_oracle_golden.py."""
    import torch
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden",
                                "cellular_4097x2049_50steps_oracle_u0.npz"))
    w = fk_inputs.workload("cellular_4097x2049", precision=precision, n_steps=50)
    assert tuple(gold["n"]) == tuple(w["n"]) and int(gold["n_steps"]) == w["n_steps"]
    plan = fk.Plan(_spec(fk, w))
    out = plan.solve()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    got = out.double().reshape(-1)[torch.tensor(gold["nodes"], device="cuda")].cpu().numpy()
    plan.close()
    assert float(gold["umax"]) == 1.0 and float(gold["umean"]) > 1e-3
    err = np.abs(got - gold["u0"]).max()
    print(f"cellular_4097x2049 {precision} vs fp64 oracle, 50 steps: max-abs {err:.3e}")
    assert err <= tol


def test_snapshots_and_resume(fk):
    """Snapshots equal the states reached by marching in chunks (fk_march)."""
    import torch
    w = _small2d(5, "fp64", n_steps=40)
    plan = fk.Plan(_spec(fk, w))
    snaps = torch.empty((4,) + plan.shape, dtype=plan.dtype, device="cuda")
    u0 = plan.solve(None, snapshots=snaps, snapshot_stride=10)
    chi = torch.tensor(fk_inputs_chi(plan.shape), dtype=plan.dtype, device="cuda")
    u = chi
    for m in range(4):
        u = plan.march(40 - 10 * m, 40 - 10 * (m + 1), u)
        assert torch.equal(u, snaps[m])
    assert torch.equal(u, u0)
    plan.close()


def fk_inputs_chi(shape):
    chi = np.zeros(shape)
    chi[0, :] = chi[-1, :] = 1.0
    chi[:, 0] = chi[:, -1] = 1.0
    return chi


@pytest.mark.parametrize("n_steps", [1, 2, 5, 6])
def test_in_place_terminal(fk, n_steps):
    import torch
    w = _small2d(4, "fp64", n_steps=n_steps)
    plan = fk.Plan(_spec(fk, w))
    u0 = torch.tensor(fk_inputs.random_field(plan.shape, seed=1), dtype=plan.dtype, device="cuda")
    ref = plan.solve(u0.clone())
    buf = u0.clone()
    plan.solve(buf, out=buf)
    assert torch.equal(buf, ref)
    plan.close()


@pytest.mark.parametrize("precision,pinned", [("fp32", True), ("fp64", False)])
def test_solve_host_buffers(fk, precision, pinned):
    """fk_solve_host (fields in host memory, copies and march enqueued on
    the stream) equals fk_solve on device buffers bit for bit: from chi, from
    a terminal field, in place, and twice in a row on the same plan; pinned
    and pageable host buffers."""
    import torch
    w = _small2d(6, precision, n_steps=30, n=(161, 81))
    plan = fk.Plan(_spec(fk, w))
    u0 = torch.tensor(fk_inputs.random_field(plan.shape, seed=5), dtype=plan.dtype)
    ref_chi = plan.solve().cpu()
    ref_u0 = plan.solve(u0.cuda()).cpu()
    torch.cuda.synchronize()

    def host(t):
        return t.pin_memory() if pinned else t
    stream = torch.cuda.current_stream()
    for _ in range(2):
        out = host(torch.full(plan.shape, float("nan"), dtype=plan.dtype))
        plan.solve_host(None, out, stream=stream)
        stream.synchronize()
        assert torch.equal(out, ref_chi)
        out = host(torch.full(plan.shape, float("nan"), dtype=plan.dtype))
        plan.solve_host(host(u0.clone()), out, stream=stream)
        stream.synchronize()
        assert torch.equal(out, ref_u0)
        buf = host(u0.clone())
        plan.solve_host(buf, buf, stream=stream)
        stream.synchronize()
        assert torch.equal(buf, ref_u0)
    assert plan.last_device_error() == 0
    assert plan.info()["workspace_bytes"] > 0
    plan.close()


@pytest.mark.parametrize("n,q,params", [
    ((3, 3), 3, (1.0, 0.2, 2 * math.pi, 0.01)),
    ((4, 3), 2, (1.0, 0.2, 2 * math.pi, 0.01)),
    ((9, 5), 8, (2.0, 0.5, 2 * math.pi, 0.5)),   # reach of many cells: halo wider than the mesh
    ((40, 3), 6, (1.0, 0.2, 2 * math.pi, 0.001)),
    ((3, 40), 6, (1.0, 0.2, 2 * math.pi, 0.001)),
])
def test_degenerate_meshes(fk, oracle, n, q, params):
    w = fk_inputs.workload("cellular_1025x513", n=n, q=q, n_steps=9, precision="fp64",
                           params=params, dt=0.01)
    got = _gpu_solve(fk, w)
    want = _oracle_march(oracle, w, 9, 0)
    assert np.abs(got - want).max() <= TOL64


def test_1d_minimal_and_wide_reach(fk, oracle, kernel1d):
    for n, dt in ((3, 1e-3), (11, 0.5)):
        w = fk_inputs.workload("bm1d_drift", n=(n,), n_steps=4, dt=dt)
        got = _gpu_solve(fk, w)
        want = _oracle_march(oracle, w, 4, 0)
        assert np.abs(got - want).max() <= TOL64


@pytest.fixture
def window_kernel(monkeypatch):
    """Plans created in the test use the window kernel where eligible."""
    monkeypatch.setenv("FK_STEP_KERNEL", "window")


@pytest.mark.parametrize("q,D", [(4, 0.02), (6, 0.02), (6, 0.005), (8, 0.01)])
def test_window_kernel_fp32_vs_oracle(fk, oracle, window_kernel, q, D):
    """FP32 window kernel (rows read once per x-point) against the oracle,
    on meshes whose band split leaves both kernels work."""
    w = fk_inputs.workload("cellular_1025x513", n=(161, 81), q=q, n_steps=100, precision="fp32",
                           params=(1.0, 0.2, 2 * math.pi, D))
    got = _gpu_solve(fk, w)
    want = _oracle_march(oracle, w, w["n_steps"], 0)
    assert np.abs(got - want).max() <= TOL32


def test_window_kernel_equals_direct(fk, monkeypatch):
    """The window and direct kernels agree to FP32 rounding on the
    benchmark workload (200 steps, random terminal field)."""
    import torch
    w = fk_inputs.workload("cellular_1025x513", n_steps=200)
    u0 = fk_inputs.random_field((513, 1025), seed=2)
    res = {}
    for kern in ("window", "direct"):
        monkeypatch.setenv("FK_STEP_KERNEL", kern)
        res[kern] = _gpu_solve(fk, w, u0)
    assert np.abs(res["window"] - res["direct"]).max() <= 2e-6


def test_window_kernel_full_march_vs_golden(fk, monkeypatch):
    monkeypatch.setenv("FK_STEP_KERNEL", "window")
    test_cellular_1025x513_fp32_full_march(fk)


# ---------------------------------------------------------------- masked window kernel
@pytest.fixture
def masked_kernel(monkeypatch):
    """Plans created in the test use the masked tensor-window kernel where eligible."""
    monkeypatch.setenv("FK_STEP_KERNEL", "masked")


# isotropic meshes on [0,2]x[0,1] (equal cell offsets on both axes), window
# widths 3..9, reach from under one cell to about three cells, so that
# exits along x, along y and along both occur on many nodes
MASKED_CASES = [
    ((81, 41), 4, 0.02, 1e-3, 4),
    ((161, 81), 6, 0.025, 1e-3, 6),
    ((161, 81), 8, 0.03, 1e-3, 8),
    ((161, 81), 8, 0.05, 1e-3, 9),
    ((161, 81), 4, 0.05, 1e-3, 6),
    ((41, 21), 6, 0.05, 1e-2, 7),
    ((33, 17), 4, 0.02, 1e-2, 4),
    ((9, 5), 4, 0.02, 1e-2, 3),
    ((5, 3), 4, 0.01, 1e-2, 3),
]


@pytest.mark.parametrize("n,q,D,dt,W", MASKED_CASES)
def test_masked_kernel_fp32_vs_oracle(fk, oracle, masked_kernel, n, q, D, dt, W):
    """Masked tensor-window kernel (exits as zero weights, every node on one
    path) against the FP64 oracle over 100 steps."""
    w = fk_inputs.workload("cellular_1025x513", n=n, q=q, n_steps=100, precision="fp32",
                           params=(1.0, 0.2, 2 * math.pi, D), dt=dt)
    got, info = _gpu_solve_info(fk, w)
    assert info["step_kernel"] == "masked" and info["window_rows"] == W
    want = _oracle_march(oracle, w, w["n_steps"], 0)
    assert np.abs(got - want).max() <= TOL32


def test_masked_kernel_const_drift(fk, oracle, masked_kernel):
    w = _small2d(4, "fp32", family="const_drift", n_steps=60, n=(81, 41))
    w.update(params=(0.7, -0.4, 0.0, 0.3))
    got, info = _gpu_solve_info(fk, w)
    assert info["step_kernel"] == "masked"
    want = _oracle_march(oracle, w, w["n_steps"], 0)
    assert np.abs(got - want).max() <= TOL32


@pytest.mark.parametrize("seed", [3, 4])
def test_masked_kernel_random_field(fk, oracle, masked_kernel, seed):
    """From a random terminal field (slopes of both signs at every face and
    corner; the end rule and the masked weights meet there)."""
    w = _small2d(6, "fp32", n=(101, 51), n_steps=5)
    u0 = fk_inputs.random_field((51, 101), seed=seed)
    got, info = _gpu_solve_info(fk, w, u0)
    assert info["step_kernel"] == "masked"
    want = _oracle_march(oracle, w, w["n_steps"], 0, u0)
    assert np.abs(got - want).max() <= TOL32


def test_masked_kernel_equals_direct(fk, monkeypatch):
    """The masked and direct kernels agree to FP32 rounding on the benchmark
    workload (200 steps, random terminal field)."""
    w = fk_inputs.workload("cellular_1025x513", n_steps=200)
    u0 = fk_inputs.random_field((513, 1025), seed=2)
    res = {}
    for kern in ("masked", "direct"):
        monkeypatch.setenv("FK_STEP_KERNEL", kern)
        res[kern], info = _gpu_solve_info(fk, w, u0)
        assert info["step_kernel"] == kern
    assert np.abs(res["masked"] - res["direct"]).max() <= 2e-6


def test_masked_kernel_full_march_vs_golden(fk, monkeypatch):
    monkeypatch.setenv("FK_STEP_KERNEL", "masked")
    test_cellular_1025x513_fp32_full_march(fk)


def test_1d_resident_snapshots_and_resume(fk):
    """The one-CTA and the cluster 1D marches: snapshots every 3 steps equal
    the per-step path's, FP32 and FP64, and a resumed march (fk_march from a
    snapshot, in place) ends where the full march does."""
    import torch
    for precision in ("fp64", "fp32"):
        w = fk_inputs.workload("bm1d_drift", n=(301,), n_steps=20, precision=precision)
        res = {}
        for kern in ("resident", "cluster", "step"):
            os.environ["FK_1D_KERNEL"] = kern
            try:
                plan = fk.Plan(_spec(fk, w))
            finally:
                os.environ.pop("FK_1D_KERNEL", None)
            u0 = torch.tensor(fk_inputs.random_field((301,), seed=5), dtype=plan.dtype,
                              device="cuda")
            snaps = torch.empty((6, 301), dtype=plan.dtype, device="cuda")
            out = plan.solve(u0, snapshots=snaps, snapshot_stride=3)
            resumed = snaps[3].clone()  # u after 12 steps, i.e. u^8
            plan.march(8, 0, resumed, out=resumed)
            torch.cuda.synchronize()
            assert plan.info()["step_kernel"] == KERNEL1D[kern]
            assert torch.equal(resumed, out)
            res[kern] = (out.double().cpu().numpy(), snaps.double().cpu().numpy())
            plan.close()
        tol = 1e-14 if precision == "fp64" else 1e-6
        for kern in ("resident", "cluster"):
            assert np.abs(res[kern][0] - res["step"][0]).max() <= tol
            assert np.abs(res[kern][1] - res["step"][1]).max() <= tol


@pytest.mark.parametrize("n,q,dt,n_steps", [
    ((201,), 8, 1e-3, 1000),   # the 1D workload in FP32
    ((1500,), 12, 1e-3, 7),
    ((3,), 8, 1e-3, 4),        # one interior node
    ((11,), 8, 0.5, 4),        # reach far beyond the mesh: most points exit
])
def test_1d_fp32_vs_oracle(fk, oracle, kernel1d, n, q, dt, n_steps):
    """FP32 1D march, one CTA for the whole march or one launch per step,
    against the FP64 oracle from a random terminal field."""
    w = fk_inputs.workload("bm1d_drift", n=n, q=q, dt=dt, n_steps=n_steps, precision="fp32")
    u0 = fk_inputs.random_field(n, seed=q)
    got, info = _gpu_solve_info(fk, w, u0)
    assert info["step_kernel"] == KERNEL1D[kernel1d]
    want = _oracle_march(oracle, w, w["n_steps"], 0, u0)
    assert np.abs(got - want).max() <= TOL32


@pytest.mark.parametrize("precision,kernel", [("fp32", "resident"), ("fp64", "cluster")])
def test_1d_default_kernel(fk, precision, kernel):
    """Without an explicit choice the 1D march runs in one launch: FP32 in
    one CTA, FP64 over a cluster."""
    w = fk_inputs.workload("bm1d_drift", precision=precision)
    _, info = _gpu_solve_info(fk, w)
    assert info["step_kernel"] == kernel
