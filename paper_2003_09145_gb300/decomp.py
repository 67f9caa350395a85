"""Slab decomposition of an Euler grid along its slowest axis, with the halo
exchange and Lax-Friedrichs speed reduction an SSP-RK3 step needs between
its stages (eq. 4.1-4.3).

Each rank stores its slab with GHOST = 3 ghost planes on either side of the
split axis (the stencil of eq. 2.4-2.6 reaches three cells).  Before every
stage the ghost planes of the stage input are filled: from the neighbouring
slabs' interior planes (periodic ends wrap around), or at a transmissive end
with copies of the boundary plane.  After the cell pass each rank holds its
slab's LF speeds as nine 64-bit words (bit patterns of non-negative doubles,
which order as integers); their maximum over ranks is the global speed of
Sec. 4's splitting (reading C7), and the CFL step (eq. dt1 / dt2 / the 3D
form) is a function of it alone, so every rank takes the same dt without a
further reduction.  The interior result then equals the undivided grid's
bit for bit.

The orchestration here is backend-agnostic: an *engine* does the local work
(the library's stage entry points on a GPU, or a restatement for CPU tests)
and a *comm* moves planes and reduces the speeds (in-process copies between
slabs, or torch.distributed point-to-point transfers and an all-reduce).

Engine interface (one slab):
    begin(Uin)                          cell pass of the stage input
    alpha_words() -> int64 tensor [9]   this slab's speeds (in place)
    end(stage, Uin, Un, Uout, t_end, dt_fixed)
    copy_planes(src, src_plane, src_packed, dst, dst_plane, dst_packed, nplanes)
    packed(nplanes) -> buffer           a packed [nvar][nplanes][plane] buffer
"""
from __future__ import annotations

from dataclasses import dataclass

GHOST = 3


def slab_bounds(n: int, nranks: int, rank: int) -> tuple[int, int]:
    """(first global plane, number of planes) of rank's slab: as even as possible."""
    base, extra = divmod(n, nranks)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


@dataclass
class SlabPlan:
    """One rank's place in the decomposition of n planes over nranks."""
    n: int
    nranks: int
    rank: int
    periodic: bool

    def __post_init__(self):
        if not 0 <= self.rank < self.nranks:
            raise ValueError("rank out of range")
        self.start, self.count = slab_bounds(self.n, self.nranks, self.rank)
        if self.count < GHOST:
            raise ValueError(f"every slab needs at least {GHOST} planes (n = {self.n}, {self.nranks} ranks)")

    @property
    def stored(self) -> int:
        """planes stored along the split axis (interior + ghosts)"""
        return self.count + 2 * GHOST

    @property
    def lower(self):
        """rank holding the planes below, or None at a non-periodic end"""
        if self.rank > 0:
            return self.rank - 1
        return self.nranks - 1 if self.periodic else None

    @property
    def upper(self):
        if self.rank < self.nranks - 1:
            return self.rank + 1
        return 0 if self.periodic else None

    # local plane indices of the four plane groups
    @property
    def lo_interior(self) -> int:
        return GHOST

    @property
    def hi_interior(self) -> int:
        return self.count

    @property
    def lo_ghost(self) -> int:
        return 0

    @property
    def hi_ghost(self) -> int:
        return self.count + GHOST


def fill_edges(engine, U, plan: SlabPlan) -> None:
    """Transmissive ends: every ghost plane takes the boundary plane (zero
    gradient, as the undivided grid's boundary treatment)."""
    if plan.lower is None:
        for g in range(GHOST):
            engine.copy_planes(U, plan.lo_interior, 0, U, plan.lo_ghost + g, 0, 1)
    if plan.upper is None:
        for g in range(GHOST):
            engine.copy_planes(U, plan.hi_interior + GHOST - 1, 0, U, plan.hi_ghost + g, 0, 1)


def exchange_local(engines, states, plans) -> None:
    """Halo exchange between slabs held in one process (one engine each)."""
    for r, (eng, U, pl) in enumerate(zip(engines, states, plans)):
        if pl.lower is not None:
            lo = plans[pl.lower]
            eng.copy_planes(states[pl.lower], lo.hi_interior, 0, U, pl.lo_ghost, 0, GHOST)
        if pl.upper is not None:
            up = plans[pl.upper]
            eng.copy_planes(states[pl.upper], up.lo_interior, 0, U, pl.hi_ghost, 0, GHOST)
        fill_edges(eng, U, pl)


class LocalGroup:
    """Several slabs in one process, advanced stage by stage together; the
    speeds are combined by an elementwise maximum over the slabs' words."""

    def __init__(self, engines, plans, maximum):
        self.engines, self.plans, self.maximum = engines, plans, maximum

    def step(self, Us, U1s, U2s, t_end=float("inf"), dt_fixed=0.0) -> None:
        for k, (ins, outs) in enumerate(((Us, U1s), (U1s, U2s), (U2s, Us)), start=1):
            exchange_local(self.engines, ins, self.plans)
            for eng, Uin in zip(self.engines, ins):
                eng.begin(Uin)
            words = [eng.alpha_words() for eng in self.engines]
            m = self.maximum(words)
            for w in words:
                w.copy_(m)
            for eng, Uin, Un, Uout in zip(self.engines, ins, Us, outs):
                eng.end(k, Uin, Un, Uout, t_end, dt_fixed)


class DistComm:
    """One slab per process: planes travel as packed buffers through
    torch.distributed point-to-point transfers (NCCL between GPUs, gloo on
    CPUs), the speeds through an all-reduce with MAX on their 64-bit words.
    Per pair of ranks the transfers match in order: every rank posts its
    sends (to the lower neighbour, then to the upper one) and its receives
    (from the upper neighbour, then from the lower one), so that even two
    ranks that are each other's lower and upper neighbour pair them right."""

    def __init__(self, dist):
        self.dist = dist

    def exchange(self, engine, U, plan: SlabPlan) -> None:
        dist = self.dist
        if plan.nranks == 1:
            if plan.periodic:
                engine.copy_planes(U, plan.hi_interior, 0, U, plan.lo_ghost, 0, GHOST)
                engine.copy_planes(U, plan.lo_interior, 0, U, plan.hi_ghost, 0, GHOST)
            fill_edges(engine, U, plan)
            return
        reqs, recvs = [], []
        if plan.lower is not None:
            b = engine.packed(GHOST)
            engine.copy_planes(U, plan.lo_interior, 0, b, 0, 1, GHOST)
            reqs.append(dist.isend(b, plan.lower))
        if plan.upper is not None:
            b = engine.packed(GHOST)
            engine.copy_planes(U, plan.hi_interior, 0, b, 0, 1, GHOST)
            reqs.append(dist.isend(b, plan.upper))
        if plan.upper is not None:
            b = engine.packed(GHOST)
            reqs.append(dist.irecv(b, plan.upper))
            recvs.append((b, plan.hi_ghost))
        if plan.lower is not None:
            b = engine.packed(GHOST)
            reqs.append(dist.irecv(b, plan.lower))
            recvs.append((b, plan.lo_ghost))
        for r in reqs:
            r.wait()
        for b, at in recvs:
            engine.copy_planes(b, 0, 1, U, at, 0, GHOST)
        fill_edges(engine, U, plan)

    def reduce_alpha(self, words) -> None:
        self.dist.all_reduce(words, op=self.dist.ReduceOp.MAX)


class SlabStepper:
    """SSP-RK3 steps of one rank's slab (U, U1, U2: stored slab states)."""

    def __init__(self, engine, plan: SlabPlan, comm: DistComm):
        self.engine, self.plan, self.comm = engine, plan, comm

    def step(self, U, U1, U2, t_end=float("inf"), dt_fixed=0.0) -> None:
        for k, (Uin, Uout) in enumerate(((U, U1), (U1, U2), (U2, U)), start=1):
            self.comm.exchange(self.engine, Uin, self.plan)
            self.engine.begin(Uin)
            self.comm.reduce_alpha(self.engine.alpha_words())
            self.engine.end(k, Uin, U, Uout, t_end, dt_fixed)
