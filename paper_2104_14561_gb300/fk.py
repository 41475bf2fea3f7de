"""PyTorch binding of the fk_* C ABI (include/fk.h).

PyTorch supplies device memory and streams; every step of the march runs
in libfk_gb300's CUDA kernels.  Fields are tensors of shape (n[1], n[0])
in 2D (x fastest), (n[2], n[1], n[0]) in 3D or (n[0],) in 1D, dtype
float32 or float64 matching the plan's precision, on the plan's CUDA
device.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L

_DTYPE = {"fp32": torch.float32, "fp64": torch.float64}
_PREC = {"fp32": L.FK_FP32, "fp64": L.FK_FP64}
_PATH = {"matrix_free": L.FK_PATH_MATRIX_FREE, "csr": L.FK_PATH_CSR}
_FAMILY = {"const_drift": L.FK_CONST_DRIFT, "cellular_flow": L.FK_CELLULAR_FLOW,
           "paper_cellular": L.FK_PAPER_CELLULAR, "runaway": L.FK_RUNAWAY_3D,
           "runaway_quench": L.FK_RUNAWAY_QUENCH_3D}


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def gauss_hermite(q: int):
    """The library's 1D Gauss-Hermite rule (density pi^{-1/2} exp(-x^2))."""
    lib = L.load()
    a = (ctypes.c_double * q)()
    w = (ctypes.c_double * q)()
    L.check("fk_gauss_hermite", lib.fk_gauss_hermite(q, a, w))
    return list(a), list(w)


def runaway_quench_params(params, t: float):
    """The runaway-model constants (E, tau, Z, delta, nu_ee, v_T, r_D, W,
    Delta_p, V_0, D_0) at time t of the thermal-quench variant with the 13
    parameters (E_0, tau, Z, T0, Tf, Ttilde, t_star, r_D, W, Delta_p, V_0,
    D_0, mc2)."""
    lib = L.load()
    q = (ctypes.c_double * 16)(*[float(v) for v in params])
    out = (ctypes.c_double * 11)()
    L.check("fk_runaway_quench_params", lib.fk_runaway_quench_params(q, float(t), out))
    return list(out)


def measure_fma_rate(precision: str = "fp32", packed: bool = False, seconds: float = 0.05,
                     stream=None) -> float:
    """FMA throughput of the current device in flop/s (2 x FMAs per second):
    the denominator of the march kernels' ALU rooflines."""
    lib = L.load()
    out = ctypes.c_double()
    L.check("fk_measure_fma_rate",
            lib.fk_measure_fma_rate(_PREC[precision], int(packed), float(seconds),
                                    ctypes.byref(out), _stream(stream)))
    return out.value


@dataclass
class PlanSpec:
    n: tuple
    lo: tuple
    hi: tuple
    family: str
    params: tuple
    q: int
    dt: float
    n_steps: int
    precision: str = "fp32"
    path: str = "matrix_free"
    periodic_x: bool = False  # x faces identified (node n[0]-1 is node 0), y faces absorb
    axes: tuple | None = None  # per axis None (uniform) or the increasing node coordinates


class Plan:
    """Owner of an fk_plan.  Create once per problem; solve many times."""

    def __init__(self, spec: PlanSpec):
        self.spec = spec
        self._lib = L.load()
        g = L.Grid()
        g.dim = len(spec.n)
        keep = []
        for m in range(g.dim):
            g.n[m] = int(spec.n[m])
            g.lo[m] = float(spec.lo[m])
            g.hi[m] = float(spec.hi[m])
            if spec.axes is not None and spec.axes[m] is not None:
                a = np.ascontiguousarray(spec.axes[m], dtype=np.float64)
                keep.append(a)
                g.axis[m] = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r = L.Region(L.FK_PERIODIC_X if spec.periodic_x else L.FK_ALL_FACES_ABSORBING)
        c = L.Coeffs()
        c.family = _FAMILY[spec.family]
        for k, v in enumerate(spec.params):
            c.p[k] = float(v)
        h = ctypes.c_void_p()
        L.check("fk_plan_create",
                self._lib.fk_plan_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(r),
                                         ctypes.byref(c), int(spec.q), float(spec.dt),
                                         int(spec.n_steps), _PREC[spec.precision],
                                         _PATH[spec.path]))
        self._h = h
        self.dtype = _DTYPE[spec.precision]
        self.shape = tuple(reversed(spec.n))
        self.device = torch.device("cuda", torch.cuda.current_device())

    # ---------------------------------------------------------------- info
    def info(self) -> dict:
        i = L.PlanInfo()
        L.check("fk_plan_get_info", self._lib.fk_plan_get_info(self._h, ctypes.byref(i)))
        return {"n_nodes": i.n_nodes, "n_interior": i.n_interior, "dim": i.dim,
                "q_per_dim": i.q_per_dim, "n_steps": i.n_steps, "halo": list(i.halo),
                "tile": list(i.tile), "reach_cells": list(i.reach_cells),
                "csr_nnz": i.csr_nnz, "workspace_bytes": i.workspace_bytes,
                "window_rows": i.window_rows,
                "step_kernel": ("direct", "window", "masked", "resident", "cluster",
                                "window3d")[i.step_kernel],
                "batch_mode": ("none", "persistent", "streams")[i.batch_mode],
                "adjoint_kernel": ("none", "scatter", "masked")[i.adjoint_kernel],
                "periodic_x": bool(i.periodic_x), "nonuniform": bool(i.nonuniform),
                "march_mode": ("steps", "persistent")[i.march_mode],
                "nodes_per_thread": i.nodes_per_thread}

    def _check_field(self, t: torch.Tensor, name: str):
        if t.dtype != self.dtype or t.device.type != "cuda" or tuple(t.shape) != self.shape \
                or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous {self.dtype} CUDA tensor of shape "
                             f"{self.shape}, got {t.dtype} {tuple(t.shape)} on {t.device}")

    def empty(self) -> torch.Tensor:
        return torch.empty(self.shape, dtype=self.dtype, device=self.device)

    # --------------------------------------------------------------- march
    def solve(self, u_terminal: torch.Tensor | None = None, out: torch.Tensor | None = None,
              snapshots: torch.Tensor | None = None, snapshot_stride: int = 0,
              stream=None) -> torch.Tensor:
        """u^0 of Scheme 1 (P(T, x) when u_terminal is None = chi)."""
        if u_terminal is not None:
            self._check_field(u_terminal, "u_terminal")
        if out is None:
            out = self.empty()
        self._check_field(out, "out")
        if snapshots is not None:
            m = self.spec.n_steps // snapshot_stride
            if snapshots.dtype != self.dtype or tuple(snapshots.shape) != (m,) + self.shape \
                    or not snapshots.is_contiguous():
                raise ValueError("snapshots: wrong dtype/shape")
        L.check("fk_solve", self._lib.fk_solve(self._h, _ptr(u_terminal), _ptr(out),
                                               _ptr(snapshots), int(snapshot_stride),
                                               _stream(stream)))
        return out

    def solve_host(self, u_terminal: torch.Tensor | None, out: torch.Tensor,
                   stream=None) -> torch.Tensor:
        """fk_solve_host: u^0 of Scheme 1 with the terminal field and the
        result in host memory (CPU tensors; pinned ones keep the copies
        asynchronous).  The copies and the march are enqueued on the stream:
        out holds u^0 once the stream has passed them."""
        for name, t in (("u_terminal", u_terminal), ("out", out)):
            if t is None:
                continue
            if t.dtype != self.dtype or t.device.type != "cpu" or \
                    tuple(t.shape) != self.shape or not t.is_contiguous():
                raise ValueError(f"{name}: expected a contiguous {self.dtype} CPU tensor of "
                                 f"shape {self.shape}, got {t.dtype} {tuple(t.shape)} on "
                                 f"{t.device}")
        if out is None:
            raise ValueError("out: a host tensor is required")
        L.check("fk_solve_host", self._lib.fk_solve_host(self._h, _ptr(u_terminal), _ptr(out),
                                                         _stream(stream)))
        return out

    def march(self, n_from: int, n_to: int, u_in: torch.Tensor,
              out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Steps n_from-1 .. n_to (resume from a checkpoint u^{n_from})."""
        self._check_field(u_in, "u_in")
        if out is None:
            out = self.empty()
        self._check_field(out, "out")
        L.check("fk_march", self._lib.fk_march(self._h, int(n_from), int(n_to), _ptr(u_in),
                                               _ptr(out), _stream(stream)))
        return out

    def solve_horizons(self, u_terminal: torch.Tensor | None = None,
                       out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Algorithm 1 (Sec. 3.2): out[k-1] = P(t_k, x) for every horizon
        t_k = k dt, k = 1..N (each a march of k steps from time t_k to 0)."""
        if u_terminal is not None:
            self._check_field(u_terminal, "u_terminal")
        shape = (self.spec.n_steps,) + self.shape
        if out is None:
            out = torch.empty(shape, dtype=self.dtype, device=self.device)
        if out.dtype != self.dtype or tuple(out.shape) != shape or not out.is_contiguous() \
                or out.device.type != "cuda":
            raise ValueError(f"out: expected a contiguous {self.dtype} CUDA tensor of shape {shape}")
        L.check("fk_solve_horizons", self._lib.fk_solve_horizons(self._h, _ptr(u_terminal),
                                                                 _ptr(out), _stream(stream)))
        return out

    def adjoint(self, cotangent_u0: torch.Tensor, u_terminal: torch.Tensor | None = None,
                checkpoint_every: int = 50, want_dtheta: bool = True,
                want_du_terminal: bool = True, stream=None):
        """dL/dtheta (4 FP64 values) and dL/du^N for L = <cotangent_u0, u^0>."""
        if cotangent_u0.dtype != torch.float64 or tuple(cotangent_u0.shape) != self.shape:
            raise ValueError("cotangent_u0 must be a float64 field")
        if u_terminal is not None:
            self._check_field(u_terminal, "u_terminal")
        dtheta = torch.zeros(4, dtype=torch.float64, device=self.device) if want_dtheta else None
        du = self.empty() if want_du_terminal else None
        L.check("fk_adjoint", self._lib.fk_adjoint(self._h, _ptr(u_terminal),
                                                   _ptr(cotangent_u0.contiguous()), _ptr(dtheta),
                                                   _ptr(du), int(checkpoint_every),
                                                   _stream(stream)))
        return dtheta, du

    def adjoint_kernel_times(self, record: bool):
        """(summed ms, launches) of the backward-step kernel over the last
        recorded adjoint call, then recording on (True) or off (False) for
        later calls (fk_adjoint_kernel_times: CUDA events around each
        launch)."""
        ms = ctypes.c_double()
        n = ctypes.c_int()
        L.check("fk_adjoint_kernel_times",
                self._lib.fk_adjoint_kernel_times(self._h, int(record), ctypes.byref(ms),
                                                  ctypes.byref(n)))
        return ms.value, n.value

    def last_device_error(self) -> int:
        return self._lib.fk_last_device_error(self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fk_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(plans, u_terminals=None, outs=None, stream=None):
    """fk_solve_batched over independent plans (one persistent launch)."""
    lib = L.load()
    n = len(plans)
    if u_terminals is None:
        u_terminals = [None] * n
    if outs is None:
        outs = [p.empty() for p in plans]
    for p, u, o in zip(plans, u_terminals, outs):
        if u is not None:
            p._check_field(u, "u_terminal")
        p._check_field(o, "out")
    H = (ctypes.c_void_p * n)(*[p._h.value for p in plans])
    U = (ctypes.c_void_p * n)(*[None if u is None else u.data_ptr() for u in u_terminals])
    O = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    L.check("fk_solve_batched", lib.fk_solve_batched(n, H, U, O, _stream(stream)))
    return outs


class ExitProbability(torch.autograd.Function):
    """u^0 = P(T, x) as a differentiable function of the coefficient
    parameters theta = p[0..3] (cellular flow: A, eps, omega, D) and of the
    terminal field.  Forward is fk_solve; backward is fk_adjoint (checkpoint
    interval `checkpoint_every`), with the parameter gradient reduced in FP64.
    """

    @staticmethod
    def forward(ctx, theta, u_terminal, spec, checkpoint_every):
        params = tuple(float(v) for v in theta.detach().cpu().tolist())
        s = PlanSpec(**{**spec.__dict__, "params": params})
        plan = Plan(s)
        ut = None if u_terminal is None else u_terminal.detach().contiguous()
        u0 = plan.solve(ut)
        ctx.plan = plan
        ctx.theta_device, ctx.theta_dtype = theta.device, theta.dtype
        ctx.ut = ut
        ctx.k = checkpoint_every
        ctx.has_ut = u_terminal is not None
        return u0

    @staticmethod
    def backward(ctx, grad_u0):
        plan = ctx.plan
        dth, du = plan.adjoint(grad_u0.detach().double().contiguous(), ctx.ut,
                               checkpoint_every=ctx.k)
        torch.cuda.current_stream().synchronize()
        plan.close()
        return (dth.to(ctx.theta_device, ctx.theta_dtype), (du if ctx.has_ut else None),
                None, None)


def exit_probability(spec: PlanSpec, theta: torch.Tensor, u_terminal: torch.Tensor | None = None,
                     checkpoint_every: int = 50) -> torch.Tensor:
    """Differentiable P(T, x) on the mesh of `spec` (its params are replaced
    by theta, a float64 tensor of 4 values)."""
    return ExitProbability.apply(theta, u_terminal, spec, checkpoint_every)
