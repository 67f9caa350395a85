"""PyTorch-facing API over the C-ABI.  Tensors are the caller's device memory;
every arithmetic step runs in the sm_103a kernels behind ``teno_*``.  PyTorch
supplies allocation and the current CUDA stream only.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib

WS_ALIGN = 256


def _stream_ptr(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _check_state(U: torch.Tensor, nvar: int, ncell: int, name: str = "U") -> None:
    if not U.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if U.dtype != torch.float64:
        raise ValueError(f"{name} must be float64")
    if not U.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if U.numel() != nvar * ncell:
        raise ValueError(f"{name} has {U.numel()} elements, expected {nvar * ncell}")


def alloc_workspace(nbytes: int, device) -> torch.Tensor:
    """Zero-filled workspace whose data pointer is 256-byte aligned."""
    raw = torch.zeros(int(nbytes) + WS_ALIGN, dtype=torch.uint8, device=device)
    off = (-raw.data_ptr()) % WS_ALIGN
    return raw[off:off + int(nbytes)]


@dataclass
class Scheme:
    """Scheme parameters of eq. 2.8, 3.1-3.2 and the gas (eq. 4.7).
    ``scheme`` selects the cutoff: "lad" (the paper's, eq. 3.1-3.4), or the
    comparison schemes "teno5" (fixed C_T = 10^-ct_m), "teno5a" (eq.
    2.16-2.18) and "wenoz" (WENO-Z weights on tau_5, eq. 2.12)."""
    gamma: float = 1.4
    H: float = 10.0
    b_l: int = 4
    b_u: int = 10
    eps: float = 1e-6
    scheme: str = "lad"
    ct_m: int = 7


class EulerGrid:
    """A uniform ndim grid of ``n`` cells (x first) with spacing ``dx`` and
    boundary types ``bc`` (0 periodic, 1 transmissive, 2 reflecting, 3 fixed
    state).  ``grav``: body acceleration of the source (0, rho g, rho u.g)
    (Sec. 4.3.2); ``bc_state``: for fixed-state axes, the conservative ghost
    state of each face, indexed [axis][side] (side 0 low, 1 high)."""

    def __init__(self, n, dx, bc, scheme: Scheme | None = None, grav=None, bc_state=None):
        self.n = tuple(int(v) for v in n)
        self.dx = tuple(float(v) for v in dx)
        self.bc = tuple(bc) if isinstance(bc, (list, tuple)) else (int(bc),) * len(self.n)
        self.scheme = scheme or Scheme()
        self.grav = tuple(float(v) for v in grav) if grav is not None else None
        self.bc_state = bc_state
        s = self.scheme
        st = None
        if bc_state is not None:
            st = [[[0.0] * 5, [0.0] * 5] for _ in range(3)]
            for k in range(len(self.n)):
                for side in range(2):
                    vals = list(bc_state[k][side]) if bc_state[k] is not None else []
                    st[k][side][:len(vals)] = [float(x) for x in vals]
        self.c = _lib.make_grid(self.n, self.dx, self.bc, s.gamma, s.H, s.b_l, s.b_u, s.eps, s.scheme, s.ct_m,
                                self.grav, st)
        self.lib = _lib.load()

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def nvar(self) -> int:
        return self.ndim + 2

    @property
    def ncell(self) -> int:
        c = 1
        for v in self.n:
            c *= v
        return c

    @property
    def state_shape(self):
        return (self.nvar,) + tuple(reversed(self.n))

    def workspace_bytes(self, op: int) -> int:
        nb = self.lib.teno_workspace_bytes(ctypes.byref(self.c), op)
        if nb == 0:
            raise ValueError("invalid grid or unsupported operation")
        return nb

    def flag_count(self) -> int:
        return int(self.lib.teno_flag_count(ctypes.byref(self.c)))


def rhs(grid: EulerGrid, U: torch.Tensor, want_flags: bool = False, ws: torch.Tensor | None = None,
        out: torch.Tensor | None = None):
    """dU/dt = L(U) (eq. 2.2) on the current CUDA stream.  Returns dUdt or
    (dUdt, flags) with the flag layout of ``teno.h``."""
    _check_state(U, grid.nvar, grid.ncell)
    dUdt = out if out is not None else torch.empty_like(U)
    flags = torch.empty(grid.flag_count(), dtype=torch.uint8, device=U.device) if want_flags else None
    if ws is None:
        ws = alloc_workspace(grid.workspace_bytes(_lib.OP_RHS), U.device)
    st = grid.lib.teno_rhs(ctypes.byref(grid.c), _ptr(U), _ptr(dUdt), _ptr(flags), _ptr(ws),
                           ws.numel(), _stream_ptr())
    _lib.check(st, "teno_rhs")
    return (dUdt, flags) if want_flags else dUdt


def device_status(ws: torch.Tensor) -> int:
    """Status recorded on the device in ``ws`` since the last query (clears it)."""
    lib = _lib.load()
    out = ctypes.c_int(0)
    _lib.check(lib.teno_get_device_status(_ptr(ws), _stream_ptr(), ctypes.byref(out)),
               "teno_get_device_status")
    return out.value


class Solver:
    """SSP-RK3 time stepper (eq. 4.1-4.3) over one grid; owns its workspace,
    the device time t and the last dt."""

    def __init__(self, grid: EulerGrid, device="cuda", cfl: float = 0.5):
        self.grid = grid
        self.device = torch.device(device)
        self.cfl = float(cfl)
        self.ws = alloc_workspace(grid.workspace_bytes(_lib.OP_RK3), self.device)
        self.t = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.dt = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.graph = None
        self._graph_key = None

    def reset_time(self, t0: float = 0.0) -> None:
        self.t.fill_(t0)

    def step(self, U: torch.Tensor, t_end: float = float("inf"), dt_fixed: float = 0.0) -> None:
        """One step in place on U: dt = dt_fixed or the CFL step, clipped to t_end."""
        g = self.grid
        _check_state(U, g.nvar, g.ncell)
        st = g.lib.teno_rk3_step(ctypes.byref(g.c), _ptr(U), self.cfl, float(dt_fixed), _ptr(self.t),
                                 float(t_end), _ptr(self.dt), _ptr(self.ws), self.ws.numel(), _stream_ptr())
        _lib.check(st, "teno_rk3_step")

    def capture(self, U: torch.Tensor, steps: int, t_end: float = float("inf"), dt_fixed: float = 0.0):
        """Capture ``steps`` RK3 steps on U into a CUDA graph (replayed by ``replay``)."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self.step(U, t_end, dt_fixed)  # warm-up outside capture
        torch.cuda.current_stream(self.device).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(steps):
                self.step(U, t_end, dt_fixed)
        self.graph = g
        self._graph_key = (U.data_ptr(), steps, t_end, dt_fixed)
        return g

    def run(self, U: torch.Tensor, t_end: float, max_steps: int = 1 << 62, dt_fixed: float = 0.0,
            chunk: int = 0) -> int:
        """Advance U to t_end (or max_steps); returns the number of steps taken.
        With chunk > 0 steps are issued ``chunk`` at a time between host checks
        of t (steps after t_end are no-ops)."""
        k = 0
        chunk = chunk or 64
        t_prev = float(self.t.item())
        while k < max_steps:
            n = min(chunk, max_steps - k)
            for _ in range(n):
                self.step(U, t_end, dt_fixed)
            k += n
            t_now = float(self.t.item())
            if t_now >= t_end:
                break
            if not t_now > t_prev:
                # no step advanced the time (dt = 0: a non-physical state,
                # which the status word reports): stop instead of spinning
                break
            t_prev = t_now
        return k

    def status(self) -> int:
        return device_status(self.ws)


class HostPipeline:
    """Advances states that live in pinned host memory, one SSP-RK3 step each:
    item k is copied to the device on an H2D stream, stepped by ``solver`` on
    the caller's current stream, and copied back on a D2H stream.  Two device
    buffers let the copy-in of item k+1 and the copy-out of item k-1 overlap
    the step of item k; CUDA events order the three streams, and no copy
    starts before run() is called (an event on the current stream).  When
    run() returns, the current stream waits for the last copy-out (nothing
    synchronises the host)."""

    def __init__(self, solver: "Solver", like: torch.Tensor):
        self.solver = solver
        dev = solver.device
        self.buf = [torch.empty(like.shape, dtype=torch.float64, device=dev) for _ in range(2)]
        self.s_in = torch.cuda.Stream(dev)
        self.s_out = torch.cuda.Stream(dev)
        self.ev_in = [torch.cuda.Event() for _ in range(2)]
        self.ev_step = [torch.cuda.Event() for _ in range(2)]
        self.ev_out = [torch.cuda.Event() for _ in range(2)]

    def run(self, host_in, host_out, t_end: float = float("inf"), dt_fixed: float = 0.0) -> None:
        """host_in[k] -> one step -> host_out[k] for every k (pinned CPU float64
        tensors shaped like the state; entries may repeat)."""
        if len(host_in) != len(host_out):
            raise ValueError("host_in and host_out differ in length")
        comp = torch.cuda.current_stream(self.solver.device)
        start = torch.cuda.Event()
        start.record(comp)
        self.s_in.wait_event(start)
        self.s_out.wait_event(start)
        used = [False, False]
        for k, (hi, ho) in enumerate(zip(host_in, host_out)):
            b = k % 2
            with torch.cuda.stream(self.s_in):
                if used[b]:
                    self.s_in.wait_event(self.ev_out[b])     # buffer b has been copied out
                self.buf[b].copy_(hi, non_blocking=True)
                self.ev_in[b].record(self.s_in)
            comp.wait_event(self.ev_in[b])
            self.solver.step(self.buf[b], t_end, dt_fixed)
            self.ev_step[b].record(comp)
            with torch.cuda.stream(self.s_out):
                self.s_out.wait_event(self.ev_step[b])
                ho.copy_(self.buf[b], non_blocking=True)
                self.ev_out[b].record(self.s_out)
            used[b] = True
        for b in range(2):
            if used[b]:
                comp.wait_event(self.ev_out[b])


class BatchSolver:
    """Many independent 1D Euler problems of uneven length (one SoA state
    U[3][sum N]) advanced together by ``teno_rk3_step_batched``: one persistent
    launch per SSP-RK3 stage, each problem with its own dx, time, final time
    and Lax-Friedrichs speeds."""

    def __init__(self, n, dx, t_end, bc: int = 1, scheme: Scheme | None = None, device="cuda",
                 cfl: float = 0.5, tuning=None):
        import numpy as np
        self.lib = _lib.load()
        self.device = torch.device(device)
        n = np.asarray(n, dtype=np.int64)
        self.nprob = int(n.size)
        self.offsets_host = np.zeros(self.nprob + 1, dtype=np.int64)
        self.offsets_host[1:] = np.cumsum(n)
        self.ncell = int(self.offsets_host[-1])
        s = scheme or Scheme()
        self.c = _lib.TenoBatch(self.nprob, self.ncell, int(bc), s.gamma, s.H, s.b_l, s.b_u, s.eps)
        self.offsets = torch.from_numpy(self.offsets_host).to(self.device)
        self.dx = torch.as_tensor(np.asarray(dx, dtype=np.float64)).to(self.device)
        self.t = torch.zeros(self.nprob, dtype=torch.float64, device=self.device)
        self.t_end = torch.as_tensor(np.asarray(t_end, dtype=np.float64)).to(self.device)
        self.cfl = float(cfl)
        nb = self.lib.teno_batch_workspace_bytes(ctypes.byref(self.c))
        if nb == 0:
            raise ValueError("invalid batch")
        self.ws = alloc_workspace(nb, self.device)
        self.set_tuning(tuning)
        offs = (ctypes.c_int64 * (self.nprob + 1))(*self.offsets_host.tolist())
        _lib.check(self.lib.teno_batch_prepare(ctypes.byref(self.c), offs, _ptr(self.ws), self.ws.numel(),
                                               _stream_ptr()), "teno_batch_prepare")
        self.graph = None

    def set_tuning(self, tuning) -> None:
        """tuning: None or (block, ctas_per_sm)."""
        self.tuning = None if tuning is None else _lib.TenoBatchTuning(int(tuning[0]), int(tuning[1]))

    def step(self, U: torch.Tensor, dt_fixed: float = 0.0) -> None:
        _check_state(U, 3, self.ncell)
        tp = ctypes.byref(self.tuning) if self.tuning is not None else None
        st = self.lib.teno_rk3_step_batched(ctypes.byref(self.c), _ptr(self.offsets), _ptr(self.dx), _ptr(U),
                                            _ptr(self.t), _ptr(self.t_end), self.cfl, float(dt_fixed), tp,
                                            _ptr(self.ws), self.ws.numel(), _stream_ptr())
        _lib.check(st, "teno_rk3_step_batched")

    def capture(self, U: torch.Tensor, steps: int, dt_fixed: float = 0.0):
        """Capture ``steps`` batched steps into a CUDA graph (``self.graph``)."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        torch.cuda.current_stream(self.device).synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(steps):
                self.step(U, dt_fixed)
        self.graph = g
        return g

    def run(self, U: torch.Tensor, max_steps: int = 1 << 62, graph_steps: int = 32) -> int:
        """Advance every problem to its t_end; graph replays of ``graph_steps``
        steps between host checks of min(t_end - t).  Returns steps issued."""
        if self.graph is None:
            self.capture(U, graph_steps)
        k = 0
        while k < max_steps:
            self.graph.replay()
            k += graph_steps
            if bool(torch.all(self.t >= self.t_end).item()):
                break
        return k

    def status(self) -> int:
        return device_status(self.ws)


SCALAR_MODES = {"lad": 0, "upwind5": 1}


class ScalarAdvection:
    """Linear advection u_t + a u_x = 0 (eq. 4.4) on a periodic 1D grid of n
    cells: the scalar form of the same TENO5-LAD reconstruction (``mode``
    "lad") or the linear weights of eq. 2.3 ("upwind5"); owns its workspace."""

    def __init__(self, n: int, dx: float, a: float = 1.0, mode: str = "lad", scheme: Scheme | None = None,
                 device="cuda"):
        self.grid = EulerGrid((n,), (dx,), (_lib.BC_PERIODIC,), scheme)
        self.a = float(a)
        self.mode = SCALAR_MODES[mode]
        self.n = int(n)
        nb = self.grid.lib.teno_scalar_workspace_bytes(ctypes.byref(self.grid.c))
        if nb == 0:
            raise ValueError("invalid scalar grid")
        self.ws = alloc_workspace(nb, torch.device(device))

    def _check(self, u: torch.Tensor) -> None:
        if u.dtype != torch.float64 or not u.is_cuda or not u.is_contiguous() or u.numel() != self.n:
            raise ValueError(f"u must be a contiguous CUDA float64 tensor of {self.n} values")

    def rhs(self, u: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """du/dt = -(f^_{i+1/2} - f^_{i-1/2}) / dx on the current stream."""
        self._check(u)
        dudt = out if out is not None else torch.empty_like(u)
        st = self.grid.lib.teno_scalar_rhs(ctypes.byref(self.grid.c), self.a, self.mode, _ptr(u), _ptr(dudt),
                                           _ptr(self.ws), self.ws.numel(), _stream_ptr())
        _lib.check(st, "teno_scalar_rhs")
        return dudt

    def step(self, u: torch.Tensor, dt: float) -> None:
        """One SSP-RK3 step (eq. 4.1-4.3) of dt, u in place."""
        self._check(u)
        st = self.grid.lib.teno_scalar_rk3_step(ctypes.byref(self.grid.c), self.a, self.mode, _ptr(u), float(dt),
                                                _ptr(self.ws), self.ws.numel(), _stream_ptr())
        _lib.check(st, "teno_scalar_rk3_step")

    def run(self, u: torch.Tensor, t_end: float, dt: float) -> int:
        """Steps of dt from t = 0 to t_end, the last one clipped; returns the count."""
        t, k = 0.0, 0
        while t < t_end:
            h = dt if t_end - t >= dt else t_end - t
            self.step(u, h)
            t += h
            k += 1
        return k


def rhs_adjoint(grid: EulerGrid, U: torch.Tensor, dUdt_bar: torch.Tensor, U_bar: torch.Tensor | None = None,
                ws: torch.Tensor | None = None) -> torch.Tensor:
    """U_bar (+)= J(U)^T dUdt_bar with the stencil selections held at their values
    for U (``teno_rhs_adjoint``).  Returns U_bar."""
    _check_state(U, grid.nvar, grid.ncell)
    _check_state(dUdt_bar, grid.nvar, grid.ncell, "dUdt_bar")
    out = torch.zeros_like(U) if U_bar is None else U_bar
    if ws is None:
        nb = grid.lib.teno_adjoint_workspace_bytes(ctypes.byref(grid.c), _lib.OP_RHS_ADJOINT)
        ws = alloc_workspace(nb, U.device)
    st = grid.lib.teno_rhs_adjoint(ctypes.byref(grid.c), _ptr(U), _ptr(dUdt_bar), _ptr(out), _ptr(ws),
                                   ws.numel(), _stream_ptr())
    _lib.check(st, "teno_rhs_adjoint")
    return out


class AdjointStepper:
    """Reverse of fixed-dt SSP-RK3 steps (``teno_rk3_step_adjoint``; with the
    step's stages U1, U2 given, ``teno_rk3_step_adjoint_staged``)."""

    def __init__(self, grid: EulerGrid, device="cuda"):
        self.grid = grid
        nb = grid.lib.teno_adjoint_workspace_bytes(ctypes.byref(grid.c), _lib.OP_RK3_ADJOINT)
        self.ws = alloc_workspace(nb, torch.device(device))

    def step(self, U_n: torch.Tensor, dt: float, Ubar_next: torch.Tensor, Ubar_n: torch.Tensor | None = None,
             stages=None):
        g = self.grid
        out = torch.empty_like(Ubar_next) if Ubar_n is None else Ubar_n
        if stages is None:
            st = g.lib.teno_rk3_step_adjoint(ctypes.byref(g.c), _ptr(U_n), float(dt), _ptr(Ubar_next), _ptr(out),
                                             _ptr(self.ws), self.ws.numel(), _stream_ptr())
            _lib.check(st, "teno_rk3_step_adjoint")
        else:
            U1, U2 = stages
            st = g.lib.teno_rk3_step_adjoint_staged(ctypes.byref(g.c), _ptr(U_n), _ptr(U1), _ptr(U2), float(dt),
                                                    _ptr(Ubar_next), _ptr(out), _ptr(self.ws), self.ws.numel(),
                                                    _stream_ptr())
            _lib.check(st, "teno_rk3_step_adjoint_staged")
        return out

    def status(self) -> int:
        return device_status(self.ws)


def rk3_step_stages(engine: "SlabEngine", U_n: torch.Tensor, dt: float):
    """One fixed-dt SSP-RK3 step from U_n through the staged entry points
    (eq. 4.1-4.3), keeping its stages: returns (U1, U2, U_next); U_n is left
    unchanged."""
    U1, U2, Un1 = torch.empty_like(U_n), torch.empty_like(U_n), torch.empty_like(U_n)
    for k, (Uin, Uout) in enumerate(((U_n, U1), (U1, U2), (U2, Un1)), start=1):
        engine.begin(Uin)
        engine.end(k, Uin, U_n, Uout, dt_fixed=dt)
    return U1, U2, Un1


class TenoRK3Rollout(torch.autograd.Function):
    """``steps`` fixed-dt SSP-RK3 steps (eq. 4.1-4.3) of the TENO5-LAD Euler
    solver as a differentiable map U0 -> U_steps.

    Forward keeps one state every ``checkpoint_every`` steps; backward replays
    each segment from its checkpoint (storing the segment's states) and runs the
    step adjoints in reverse.  With ``keep_stages`` the replay also keeps each
    step's stages U1, U2 (three states per step of a segment) and the step
    adjoints take them (``teno_rk3_step_adjoint_staged``); otherwise they are
    recomputed inside ``teno_rk3_step_adjoint``.  Both give the same gradient
    bit for bit."""

    @staticmethod
    def forward(ctx, U0: torch.Tensor, grid: EulerGrid, steps: int, dt: float, checkpoint_every: int = 0,
                keep_stages: bool = True):
        k = checkpoint_every if checkpoint_every > 0 else max(1, int(round(steps ** 0.5)))
        solver = Solver(grid, device=U0.device)
        U = U0.detach().clone()
        ckpts = {0: U.clone()}
        for n in range(steps):
            solver.step(U, float("inf"), dt_fixed=dt)
            if (n + 1) % k == 0 and n + 1 < steps:
                ckpts[n + 1] = U.clone()
        ctx.grid, ctx.steps, ctx.dt, ctx.k, ctx.ckpts, ctx.solver = grid, steps, dt, k, ckpts, solver
        ctx.keep_stages = bool(keep_stages)
        return U

    @staticmethod
    def backward(ctx, Ubar: torch.Tensor):
        grid, steps, dt, k = ctx.grid, ctx.steps, ctx.dt, ctx.k
        adj = AdjointStepper(grid, device=Ubar.device)
        solver = ctx.solver
        engine = SlabEngine(grid, device=Ubar.device) if ctx.keep_stages else None
        B = Ubar.detach().contiguous().clone()
        seg_starts = sorted(ctx.ckpts)
        for s0 in reversed(seg_starts):
            s1 = min(s0 + k, steps)
            states, stages = [ctx.ckpts[s0].clone()], []
            for _ in range(s0, s1):
                if engine is not None:
                    U1, U2, Un1 = rk3_step_stages(engine, states[-1], dt)
                    stages.append((U1, U2))
                    states.append(Un1)
                elif len(states) < s1 - s0:
                    U = states[-1].clone()
                    solver.step(U, float("inf"), dt_fixed=dt)
                    states.append(U)
            for n in range(s1 - 1, s0 - 1, -1):
                adj.step(states[n - s0], dt, B, B, stages=stages[n - s0] if engine is not None else None)
            del states, stages
        return B, None, None, None, None, None


def rollout(U0: torch.Tensor, grid: EulerGrid, steps: int, dt: float, checkpoint_every: int = 0,
            keep_stages: bool = True) -> torch.Tensor:
    """Differentiable fixed-dt rollout (see TenoRK3Rollout)."""
    return TenoRK3Rollout.apply(U0, grid, steps, dt, checkpoint_every, keep_stages)


# ----------------------------------------------------------------------------
# Domain decomposition along the slowest axis (decomp.py): the GPU engine
# ----------------------------------------------------------------------------

def slab_grid(grid: EulerGrid, plan) -> EulerGrid:
    """The stored grid of one slab of ``grid``: plan.stored planes along the
    slowest axis (interior + 3 ghost planes per side), transmissive there
    (the ghost planes carry the neighbours' or the boundary's data)."""
    from . import decomp
    ax = grid.ndim - 1
    if plan.n != grid.n[ax]:
        raise ValueError("plan does not match the grid")
    n = list(grid.n)
    n[ax] = plan.stored
    bc = list(grid.bc)
    if bc[ax] not in (_lib.BC_PERIODIC, _lib.BC_TRANSMISSIVE):
        raise ValueError("the split axis must be periodic or transmissive")
    bc[ax] = _lib.BC_TRANSMISSIVE
    assert decomp.GHOST == 3
    return EulerGrid(tuple(n), grid.dx, tuple(bc), grid.scheme, grid.grav, grid.bc_state)


def slab_from_global(U: torch.Tensor, grid: EulerGrid, plan) -> torch.Tensor:
    """A stored slab state (ghost planes zero) holding plan's planes of U."""
    from .decomp import GHOST
    shape = (grid.nvar,) + tuple(reversed(grid.n))
    Ug = U.reshape(shape)
    out = torch.zeros((grid.nvar, plan.stored) + shape[2:], dtype=U.dtype, device=U.device)
    out[:, GHOST:GHOST + plan.count] = Ug[:, plan.start:plan.start + plan.count]
    return out.reshape(-1)


def slab_interior(Us: torch.Tensor, grid: EulerGrid, plan) -> torch.Tensor:
    """The interior planes of a stored slab state, shaped like U's slice."""
    from .decomp import GHOST
    shape = (grid.nvar, plan.stored) + tuple(reversed(grid.n))[1:]
    return Us.reshape(shape)[:, GHOST:GHOST + plan.count]


class SlabEngine:
    """decomp.py's engine for one slab on a GPU: the staged SSP-RK3 entry
    points (teno_rk3_stage_begin / _end), the LF-speed words of its
    workspace, and plane copies (teno_planes_copy)."""

    def __init__(self, grid: EulerGrid, device="cuda", cfl: float = 0.5):
        self.grid = grid
        self.device = torch.device(device)
        self.cfl = float(cfl)
        self.ws = alloc_workspace(grid.workspace_bytes(_lib.OP_RK3), self.device)
        off = int(grid.lib.teno_alpha_offset())
        self._alpha = self.ws[off:off + 9 * 8].view(torch.int64)
        self.t = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.dt = torch.zeros(1, dtype=torch.float64, device=self.device)
        ax = grid.ndim - 1
        self.plane = grid.ncell // grid.n[ax]

    def begin(self, Uin: torch.Tensor) -> None:
        g = self.grid
        _check_state(Uin, g.nvar, g.ncell, "Uin")
        _lib.check(g.lib.teno_rk3_stage_begin(ctypes.byref(g.c), _ptr(Uin), _ptr(self.ws), self.ws.numel(),
                                              _stream_ptr()), "teno_rk3_stage_begin")

    def alpha_words(self) -> torch.Tensor:
        return self._alpha

    def end(self, stage: int, Uin, Un, Uout, t_end: float = float("inf"), dt_fixed: float = 0.0) -> None:
        g = self.grid
        _lib.check(g.lib.teno_rk3_stage_end(ctypes.byref(g.c), int(stage), _ptr(Uin), _ptr(Un), _ptr(Uout),
                                            self.cfl, float(dt_fixed), _ptr(self.t), float(t_end), _ptr(self.dt),
                                            _ptr(self.ws), self.ws.numel(), _stream_ptr()), "teno_rk3_stage_end")

    def copy_planes(self, src, src_plane, src_packed, dst, dst_plane, dst_packed, nplanes) -> None:
        g = self.grid
        _lib.check(g.lib.teno_planes_copy(ctypes.byref(g.c), _ptr(src), int(src_plane), int(src_packed), _ptr(dst),
                                          int(dst_plane), int(dst_packed), int(nplanes), _stream_ptr()),
                   "teno_planes_copy")

    def packed(self, nplanes: int) -> torch.Tensor:
        return torch.empty(self.grid.nvar * nplanes * self.plane, dtype=torch.float64, device=self.device)

    def status(self) -> int:
        return device_status(self.ws)
