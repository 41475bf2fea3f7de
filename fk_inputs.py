"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds workload definitions (mesh sizes, coefficient parameters,
step counts) and seeded random-number recipes only.  It contains none of the
method's arithmetic, and neither the oracle nor the CUDA path is imported
here.

Workloads (the paper has no datasets; every input is defined by formulas):

* ``bm1d_drift``           -- 1D Brownian motion with drift b = 0.5, sigma = 1
                              on (-1, 1), T = 1, 201 nodes, 8 Gauss-Hermite
                              points, dt = 1e-3 (1000 steps), FP64, terminal
                              field chi (Sec. 4.1 with drift).
* ``cellular_1025x513``    -- passive tracer in the time-periodic cellular
                              flow psi = A sin(pi x) sin(pi y)
                              + eps sin(omega t) sin(2 pi x) sin(pi y), A = 1,
                              eps = 0.2, omega = 2 pi, D = 1e-3, box
                              [0,2] x [0,1], 1025 x 513 nodes, 6 x 6 points,
                              dt = 1e-3, 2000 steps (T = 2), FP32 (Sec. 4.2
                              family, our stream-function form).
* ``cellular_4097x2049``   -- the same flow, 4097 x 2049, 8 x 8 points,
                              dt = 5e-4, 4000 steps, FP32 and FP64.
* ``cellular_autonomous_2049x1025`` -- eps = 0, 2049 x 1025, 8 x 8 points,
                              dt = 5e-4, 4000 steps, assembled-CSR path.
* ``batched_64``           -- 64 instances: nx odd uniform in [257, 2049],
                              ny = (nx+1)/2, D = 10^U[-4,-2], A ~ U[0.5, 2],
                              eps = 0.2, omega = 2 pi, 6 x 6 points,
                              dt = 1e-3, 1000 steps, FP32, fixed seed.
* ``adjoint_1025x513``     -- the 1025 x 513 workload differentiated with
                              respect to A, eps, D and the terminal field.
* ``paper_2d_1025x257``    -- the paper's own 2D example (Sec. 4.2): Pe = 10,
                              n = 2, eps = 0.15, omega = 2 pi / 10 on
                              [-pi, pi] x [0, 1], periodic in x, 6 x 6
                              points, dt = 5e-5, 1000 steps (T = 0.05), FP32.
* ``graded_1025x513``      -- the cellular_1025x513 problem on a mesh graded
                              towards every face (non-uniform axes).
* ``horizons_1025x513``    -- every horizon t_k = k dt, k = 1..200, of the
                              cellular flow (Algorithm 1).
* ``runaway_97x65x41``     -- the runaway-electron model of Sec. 4.3 at the
                              paper's parameters on (2, 50) x (-1, 1) x
                              (0, 1), 97 x 65 x 41 nodes, 4 x 4 x 4 points,
                              dt = 5e-3, 4800 steps (T = 24), FP32.
* ``drift3d_129``          -- d = 3: Brownian motion with drift
                              b = (0.3, -0.2, 0.1), sigma = 0.5 in (-1, 1)^3,
                              129^3 nodes, 4 x 4 x 4 points, dt = 1e-3,
                              500 steps (T = 0.5), FP32.

Values in every workload are probabilities in [0, 1] that start from the 0/1
indicator chi with a sharp ramp at the boundary; ``random_field`` draws
fields of that kind for single-step checks.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi

WORKLOADS = {
    "bm1d_drift": dict(n=(201,), lo=(-1.0,), hi=(1.0,), family="const_drift",
                       params=(0.5, 0.0, 0.0, 1.0), q=8, dt=1e-3, n_steps=1000,
                       precision="fp64"),
    "cellular_1025x513": dict(n=(1025, 513), lo=(0.0, 0.0), hi=(2.0, 1.0),
                              family="cellular_flow", params=(1.0, 0.2, TWO_PI, 1e-3),
                              q=6, dt=1e-3, n_steps=2000, precision="fp32"),
    "cellular_4097x2049": dict(n=(4097, 2049), lo=(0.0, 0.0), hi=(2.0, 1.0),
                               family="cellular_flow", params=(1.0, 0.2, TWO_PI, 1e-3),
                               q=8, dt=5e-4, n_steps=4000, precision="fp32"),
    "cellular_autonomous_2049x1025": dict(n=(2049, 1025), lo=(0.0, 0.0), hi=(2.0, 1.0),
                                          family="cellular_flow",
                                          params=(1.0, 0.0, TWO_PI, 1e-3), q=8, dt=5e-4,
                                          n_steps=4000, precision="fp32", path="csr"),
    "adjoint_1025x513": dict(n=(1025, 513), lo=(0.0, 0.0), hi=(2.0, 1.0),
                             family="cellular_flow", params=(1.0, 0.2, TWO_PI, 1e-3),
                             q=6, dt=1e-3, n_steps=2000, precision="fp32"),
    # the paper's own example (Sec. 4.2): Pe = 10, n = 2, eps = 0.15,
    # omega = 2 pi / 10, T = 0.05 on [-pi, pi] x [0, 1], periodic in x
    "paper_2d_1025x257": dict(n=(1025, 257), lo=(-math.pi, 0.0), hi=(math.pi, 1.0),
                              family="paper_cellular", params=(10.0, 2.0, 0.15, TWO_PI / 10),
                              q=6, dt=5e-5, n_steps=1000, precision="fp32", periodic_x=True),
    # the benchmark flow on a mesh graded towards every face (non-uniform
    # axes: spacing 2x finer at the faces than in the middle)
    "graded_1025x513": dict(n=(1025, 513), lo=(0.0, 0.0), hi=(2.0, 1.0),
                            family="cellular_flow", params=(1.0, 0.2, TWO_PI, 1e-3),
                            q=6, dt=1e-3, n_steps=2000, precision="fp32", graded=(0.4, 0.4)),
    # d = 3: Brownian motion with constant drift in the cube (-1, 1)^3
    # (independent components, so the survival is a product of 1D ones)
    "drift3d_129": dict(n=(129, 129, 129), lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0),
                        family="const_drift", params=(0.3, -0.2, 0.1, 0.5), q=4, dt=1e-3,
                        n_steps=500, precision="fp32"),
    # the runaway-electron model of Sec. 4.3 at the paper's parameters,
    # p in (2, 50), xi in (-1, 1), r in (0, 1), uniform mesh, T = 24 (the
    # first time of the paper's figures)
    "runaway_97x65x41": dict(n=(97, 65, 41), lo=(2.0, -1.0, 0.0), hi=(50.0, 1.0, 1.0),
                             family="runaway",
                             params=(0.3, 1e5, 1.0, 0.042, 1.0, 1.0, 0.7, 1e-2, 20.0, 0.003,
                                     1e-4),
                             q=4, dt=5e-3, n_steps=4800, precision="fp32"),
    # the thermal-quench variant at the end of Sec. 4.3 at the constants the
    # paper prints there (E_0 = 1e-3, tau = 6000, Z = 1, T0 = 3, Tf = 0.005,
    # Ttilde = 3 keV, r_D = 0, W = 1e-4, Delta_p = 2, V_0 = 0) with the free
    # pair D_0 = 0.01 (the value of the paper's figure) and t_star = 2, mc2 =
    # 511 keV; the static model's box, T = 12.  As the plasma cools the
    # collision rates grow as T^{-3/2} (pitch-angle scattering reaches
    # sigma_xi ~ 1.9), so the xi axis has 33 nodes and dt = 1e-3 to keep
    # every shifted point within the 3D node window
    "runaway_quench_97x33x41": dict(n=(97, 33, 41), lo=(2.0, -1.0, 0.0), hi=(50.0, 1.0, 1.0),
                                    family="runaway_quench",
                                    params=(1e-3, 6000.0, 1.0, 3.0, 0.005, 3.0, 2.0, 0.0, 1e-4,
                                            2.0, 0.0, 0.01, 511.0),
                                    q=4, dt=1e-3, n_steps=12000, precision="fp32"),
    # the same model on the paper's non-uniform radial grid (Sec. 4.3): r
    # spaced 0.1 on [0, r_D] and 0.0025 on [r_D, 1] (7 + 120 cells), which
    # resolves the boundary layer at r_D = 0.7
    "runaway_nonuniform_97x65x128": dict(
        n=(97, 65, 128), lo=(2.0, -1.0, 0.0), hi=(50.0, 1.0, 1.0), family="runaway",
        params=(0.3, 1e5, 1.0, 0.042, 1.0, 1.0, 0.7, 1e-2, 20.0, 0.003, 1e-4),
        q=4, dt=5e-3, n_steps=4800, precision="fp32", r_axis=(0.7, 0.1, 0.0025)),
    # every horizon t_k = k dt, k = 1..200, of the time-dependent flow (Algorithm 1)
    "horizons_1025x513": dict(n=(1025, 513), lo=(0.0, 0.0), hi=(2.0, 1.0),
                              family="cellular_flow", params=(1.0, 0.2, TWO_PI, 1e-3),
                              q=6, dt=1e-3, n_steps=200, precision="fp32"),
}

BATCH_SEED = 20240214


def graded_axis(lo: float, hi: float, n: int, strength: float) -> np.ndarray:
    """n increasing coordinates on [lo, hi] clustered towards both ends: a
    uniform grid xi in [-1, 1] mapped by (1 - s) xi + s sin(pi xi / 2)."""
    xi = np.linspace(-1.0, 1.0, n)
    t = (1.0 - strength) * xi + strength * np.sin(0.5 * math.pi * xi)
    x = 0.5 * (lo + hi) + 0.5 * (hi - lo) * t
    x[0], x[-1] = lo, hi
    return x


def two_spacing_axis(lo: float, mid: float, hi: float, coarse: float, fine: float) -> np.ndarray:
    """Coordinates spaced `coarse` on [lo, mid] and `fine` on [mid, hi] (the
    shape of the paper's non-uniform radial grid of Sec. 4.3)."""
    a = lo + np.arange(0, int(round((mid - lo) / coarse))) * coarse
    b = mid + np.arange(0, int(round((hi - mid) / fine)) + 1) * fine
    x = np.concatenate([a, b])
    x[0], x[-1] = lo, hi
    return x


def axes_of(w: dict):
    """The node coordinates of a workload with graded or explicit axes, else
    None (uniform)."""
    if w.get("axes") is not None:
        return tuple(None if a is None else np.asarray(a, dtype=np.float64) for a in w["axes"])
    if not w.get("graded"):
        return None
    return tuple(graded_axis(w["lo"][m], w["hi"][m], w["n"][m], w["graded"][m])
                 for m in range(len(w["n"])))


def workload(name: str, **override) -> dict:
    w = dict(WORKLOADS[name])
    w.setdefault("path", "matrix_free")
    w.update(override)
    if w.get("r_axis") and w.get("axes") is None:
        mid, coarse, fine = w["r_axis"]
        r = two_spacing_axis(w["lo"][2], mid, w["hi"][2], coarse, fine)
        assert len(r) == w["n"][2], (len(r), w["n"][2])
        w["axes"] = (None, None, r)
    return w


def batched_instances(count: int = 64, seed: int = BATCH_SEED, nx_range=(257, 2049)):
    """Grids and parameters of the batched sweep: nx odd and uniform in
    nx_range, ny = (nx+1)/2 (square cells on [0,2] x [0,1]), D log-uniform in
    [1e-4, 1e-2], A uniform in [0.5, 2]."""
    rng = np.random.default_rng(seed)
    out = []
    lo_h, hi_h = (nx_range[0] - 1) // 2, (nx_range[1] - 1) // 2
    for _ in range(count):
        nx = 2 * int(rng.integers(lo_h, hi_h + 1)) + 1
        ny = (nx + 1) // 2
        D = 10.0 ** rng.uniform(-4.0, -2.0)
        A = rng.uniform(0.5, 2.0)
        out.append(dict(n=(nx, ny), lo=(0.0, 0.0), hi=(2.0, 1.0), family="cellular_flow",
                        params=(A, 0.2, TWO_PI, D), q=6, dt=1e-3, n_steps=1000,
                        precision="fp32"))
    return out


# batched workloads: the 64-instance sweep, and a launch-bound batch of 256
# small instances (nx in [33, 129]) drawn the same way
BATCHES = {"batched_64": dict(count=64, nx_range=(257, 2049)),
           "batched_small_256": dict(count=256, nx_range=(33, 129))}


def batch(name: str):
    """The instances of a named batched workload."""
    return batched_instances(**BATCHES[name])


def random_field(shape, seed: int, modes: int = 6, boundary_one: bool = True) -> np.ndarray:
    """A smooth seeded field with values in [0, 1]: a random combination of
    low Fourier modes passed through a logistic squash, boundary nodes set to
    1 (as every march state has), plus a few sharp ramps."""
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.linspace(0.0, 1.0, s) for s in shape], indexing="ij")
    f = np.zeros(shape)
    for _ in range(modes):
        k = rng.integers(1, 6, size=len(shape))
        ph = rng.uniform(0, 2 * math.pi, size=len(shape))
        term = np.ones(shape)
        for g, kk, pp in zip(grids, k, ph):
            term = term * np.cos(math.pi * kk * g + pp)
        f += rng.normal() * term
    f = 1.0 / (1.0 + np.exp(-2.0 * f))
    if boundary_one:
        for ax in range(len(shape)):
            sl = [slice(None)] * len(shape)
            sl[ax] = 0
            f[tuple(sl)] = 1.0
            sl[ax] = -1
            f[tuple(sl)] = 1.0
    return f


def sample_nodes(shape, count: int, seed: int) -> np.ndarray:
    """Seeded flat node indices, always including the corners and the
    nodes next to the boundary."""
    rng = np.random.default_rng(seed)
    J = int(np.prod(shape))
    pick = set(rng.integers(0, J, size=count).tolist())
    if len(shape) == 2:
        ny, nx = shape
        for k in (0, 1, ny // 2, ny - 2, ny - 1):
            for i in (0, 1, nx // 2, nx - 2, nx - 1):
                pick.add(k * nx + i)
    if len(shape) == 3:
        nz, ny, nx = shape
        for l in (0, 1, nz // 2, nz - 2, nz - 1):
            for k in (0, 1, ny // 2, ny - 2, ny - 1):
                for i in (0, 1, nx // 2, nx - 2, nx - 1):
                    pick.add((l * ny + k) * nx + i)
    return np.array(sorted(pick), dtype=np.int64)
