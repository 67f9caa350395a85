"""The slab decomposition's host orchestration (paper_2003_09145_gb300/decomp.py)
on CPU: plans, and world-size 2 and 3 gloo runs whose local stages are the
oracle's (test infrastructure), against the oracle's undivided run.

Each rank stores its slab with three ghost planes per side; before every
SSP-RK3 stage (eq. 4.1-4.3) the ghost planes are exchanged (periodic ends
wrap, transmissive ends copy the boundary plane), the Lax-Friedrichs speeds
are all-reduced with MAX on their 64-bit words (Sec. 4, reading C7), and the
CFL step (eq. dt1 / dt2 / 3D) follows from them on every rank alike.  The
interior of every slab must equal the undivided run bit for bit."""
import os
import socket
import struct
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2003_09145_gb300 import decomp  # noqa: E402


def test_slab_plans():
    for n, R in ((18, 2), (19, 3), (40, 4), (7, 2)):
        spans = [decomp.slab_bounds(n, R, r) for r in range(R)]
        assert spans[0][0] == 0 and sum(c for _, c in spans) == n
        assert all(spans[r][0] + spans[r][1] == spans[r + 1][0] for r in range(R - 1))
        assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    p = decomp.SlabPlan(20, 4, 0, periodic=True)
    assert (p.lower, p.upper, p.stored) == (3, 1, 11)
    q = decomp.SlabPlan(20, 4, 3, periodic=False)
    assert (q.lower, q.upper) == (2, None)
    assert (q.lo_ghost, q.lo_interior, q.hi_interior, q.hi_ghost) == (0, 3, 5, 8)
    with pytest.raises(ValueError):
        decomp.SlabPlan(5, 3, 0, periodic=True)     # slabs thinner than the stencil's reach


class OracleSlabEngine:
    """decomp.py's engine on CPU with the oracle doing the local work: the LF
    speeds of the stored slab, and each stage's right-hand side at the
    interior cells under the all-reduced speeds, combined as the oracle's
    RK3 step combines them."""

    def __init__(self, oracle, n, dx, bc, plan, cfl):
        self.o = oracle
        self.n, self.dx, self.bc, self.plan, self.cfl = n, dx, bc, plan, cfl
        self.ndim = len(n)
        self.nvar = self.ndim + 2
        self.plane = int(np.prod(n[:-1])) if self.ndim > 1 else 1
        self.words = torch.zeros(9, dtype=torch.int64)
        g = decomp.GHOST
        self.cells = np.arange(g * self.plane, (g + plan.count) * self.plane)
        self.t, self.dt = 0.0, 0.0

    def _view(self, U):
        return U.numpy().reshape(self.nvar, -1)

    def begin(self, Uin):
        w = np.zeros(9, dtype=np.int64)
        for d in range(self.ndim):
            a = self.o.lf_alpha(self.ndim, self.n, d, Uin.numpy())
            for s, f in enumerate((0, 1, self.nvar - 1)):
                w[3 * d + s] = struct.unpack("<q", struct.pack("<d", a[f]))[0]
        self.words.copy_(torch.from_numpy(w))

    def alpha_words(self):
        return self.words

    def end(self, stage, Uin, Un, Uout, t_end, dt_fixed):
        w = self.words.numpy()
        sp = np.array([[struct.unpack("<d", struct.pack("<q", int(w[3 * d + s])))[0] for s in range(3)]
                       for d in range(self.ndim)])
        alpha = np.array([[a[0]] + [a[1]] * self.ndim + [a[2]] for a in sp])
        if stage == 1:
            smax = [max(a[0], a[2]) for a in sp]        # max(|u| + c) = max(max|u-c|, max|u+c|)
            dx = self.dx
            if self.ndim == 1:
                dt = self.cfl * dx[0] / smax[0]
            elif self.ndim == 2:
                dtx, dty = dx[0] / smax[0], dx[1] / smax[1]
                dt = self.cfl * dtx * dty / (dtx + dty)
            else:
                acc = 0.0
                for d in range(3):
                    acc += smax[d] / dx[d]
                dt = self.cfl / acc
            self.dt = min(dt, t_end - self.t)
            self.t += self.dt
        L = self.o.euler_rhs_sample(Uin.numpy(), self.n, self.dx, self.bc, self.cells, alpha=alpha).T
        c, dt = self.cells, self.dt
        un, uk, uo = self._view(Un), self._view(Uin), self._view(Uout)
        if stage == 1:
            uo[:, c] = un[:, c] + dt * L
        elif stage == 2:
            uo[:, c] = 3.0 / 4.0 * un[:, c] + 1.0 / 4.0 * uk[:, c] + 1.0 / 4.0 * dt * L
        else:
            uo[:, c] = 1.0 / 3.0 * un[:, c] + 2.0 / 3.0 * uk[:, c] + 2.0 / 3.0 * dt * L

    def copy_planes(self, src, sp, spk, dst, dp, dpk, nplanes):
        a = src.numpy().reshape(self.nvar, -1, self.plane)
        b = dst.numpy().reshape(self.nvar, -1, self.plane)
        b[:, (0 if dpk else dp):(0 if dpk else dp) + nplanes] = a[:, (0 if spk else sp):(0 if spk else sp) + nplanes]

    def packed(self, nplanes):
        return torch.empty(self.nvar * nplanes * self.plane, dtype=torch.float64)


def _case(name):
    from paper_2003_09145_gb300 import inputs
    if name == "3d-periodic":
        n = (6, 5, 12)
        return inputs.random_smooth_state(3, n, seed=4, amp=0.05), n, (0.2, 0.25, 0.15), (0, 0, 0)
    if name == "2d-transmissive":
        n = (8, 15)
        return inputs.random_discontinuous_state(2, n, seed=6), n, (0.1, 0.08), (0, 1)
    n = (31,)
    return inputs.random_discontinuous_state(1, n, seed=8), n, (0.05,), (1,)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, case, steps, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    import oracle
    from paper_2003_09145_gb300 import decomp as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    U0, n, dx, bc = _case(case)
    ax = len(n) - 1
    plan = D.SlabPlan(n[ax], world, rank, periodic=(bc[ax] == 0))
    nloc = list(n)
    nloc[ax] = plan.stored
    bloc = list(bc)
    bloc[ax] = 1
    eng = OracleSlabEngine(oracle, tuple(nloc), dx, tuple(bloc), plan, 0.5)
    nvar = len(n) + 2
    Ug = U0.reshape((nvar, n[ax], -1))
    loc = np.zeros((nvar, plan.stored, Ug.shape[2]))
    loc[:, D.GHOST:D.GHOST + plan.count] = Ug[:, plan.start:plan.start + plan.count]
    U = torch.from_numpy(loc.reshape(-1).copy())
    U1, U2 = torch.zeros_like(U), torch.zeros_like(U)
    stepper = D.SlabStepper(eng, plan, D.DistComm(dist))
    dts = []
    for _ in range(steps):
        stepper.step(U, U1, U2)
        dts.append(eng.dt)
    interior = U.numpy().reshape(nvar, plan.stored, -1)[:, D.GHOST:D.GHOST + plan.count].copy()
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, plan.start, interior, dts))


@pytest.mark.parametrize("case,world,steps", [("3d-periodic", 2, 3), ("2d-transmissive", 3, 3),
                                              ("1d-transmissive", 2, 4)])
def test_gloo_ranks_equal_undivided_oracle(oracle, case, world, steps):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    U0, n, dx, bc = _case(case)
    nvar = len(n) + 2
    ref = np.array(U0)
    ref_dts = []
    t = 0.0
    for _ in range(steps):
        ref, t2, k = oracle.euler_run(ref, n, dx, bc, float("inf"), sigma=0.5, max_steps=1, t0=t)
        ref_dts.append(t2 - t)
        t = t2
    Rg = ref.reshape((nvar, n[-1], -1))
    for rank, start, interior, dts in res:
        np.testing.assert_array_equal(interior, Rg[:, start:start + interior.shape[1]])
        np.testing.assert_allclose(dts, ref_dts, rtol=1e-12)
