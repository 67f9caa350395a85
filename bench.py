"""Benchmark: SSP-RK3 steps of the TENO5-LAD Euler solver on the 3D periodic
turbulence box (256^3 cells, FP64), reported in Gcell-updates/s (one cell
advanced one full RK3 step = three right-hand-side evaluations).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 (torchrun) runs N independent replicas,
one per GPU, with no data exchange ("replicas only"); the timed region is
bracketed by a barrier and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RHS Gcell-updates/s & roofline fraction; batched/adjoint vs plain at 1e-10"
UNIT = "Gcell-updates/s"
WORKLOAD = ("3D periodic compressible Euler, random-phase solenoidal velocity E(k)~k^4 exp(-2(k/4)^2), "
            "Mt 0.6, 256^3 cells, TENO5-LAD + global LF + characteristic projection, SSP-RK3 CFL 0.5")
N_CELLS_1D = 256
SM_COUNT = 152
FP64_FLOP_PER_CLK_PER_SM = 4          # 2 FP64 FMA lanes per SM per clock
# Algorithmic FP64 work of one interface flux at nvar = 5 (3D), counting the
# formulas the kernel evaluates in binary64 (add/mul = 1 flop, FMA = 2,
# divide / rsqrt = 1).
# * Every stencil kept at all ten reconstructions (certified in FP32): the
#   closed form F~ + a_mid U~ + acoustic corrections -- Roe average 25 (from
#   the cell pass's m/sqrt(rho): 1/(sr_a + sr_b), u~ 6, |u~|^2 5, H~ 2,
#   c^2 3, rsqrt, c, the halved coefficients 5), per point 20 (the
#   P-weighted sum of the cell pass's F/2 and the M-weighted sum of U),
#   l_0.U~ and l_E.U~ as A +- B 12, the combined corrections 6 and the
#   output 24: 187.  (Forming F_d/2 costs 5 flops per cell and direction in
#   the cell pass, plus E + p once; its mass component m_d/2 is not formed:
#   the P-weighted sum takes m_d itself.)  The weighted sums are counted at
#   one multiply-add per point and component.  The kernel keeps them in
#   integer weights; it evaluates the five M-weighted sums and the mass
#   component's P-weighted sum in 64-bit fixed point on the integer pipes
#   (exact terms, one rounding: teno_fixsum.cuh) and the other four
#   P-weighted sums as binary64 chains that skip the products with weights
#   +-1 (9 of their 12 flops), so 187 - 6 x 12 - 4 x 3 = 103 flops per
#   interface run on the FP64 pipe: fp64_flops_per_interface.  The roofline keeps the
#   algorithmic count against the FP64 peak, the rate at which binary64
#   could evaluate the same arithmetic.
# * Otherwise the characteristic path: Roe 27, projection 6 x 20, split 6 x 28,
#   sum 5, back-projection 21 (= 341), plus per scalar reconstruction 9 when
#   its own FP32 pre-test keeps every stencil, else 38 for the binary64
#   indicators, m and weights plus 21 for the cutoff test.
def alg_counts(ndim: int):
    """(closed form, characteristic path) algorithmic FP64 flops per interface
    for an ndim grid, term by term as listed above (D = ndim, nvar = D + 2):
    closed = Roe (2 + 2D + (2D - 1) + 2 + 3 + 1 + 1 + 5) + 6 points x 4 nvar
             + A +- B (2D + 6) + corrections 6 + output (4D + 12);
    characteristic = Roe (the same + b1 and u_d/2: 2) + 6 x projection (4D + 8)
             + 6 x split (22 + 3 (D - 1)) + sum nvar + back-projection
             (13 + 4 (D - 1)).  3D: 187 and 341; 2D: 153 and 290."""
    D, nv = ndim, ndim + 2
    roe = 2 + 2 * D + (2 * D - 1) + 2 + 3 + 1 + 1 + 5
    closed = roe + 6 * 4 * nv + (2 * D + 6) + 6 + (4 * D + 12)
    char = roe + 2 + 6 * (4 * D + 8) + 6 * (22 + 3 * (D - 1)) + nv + (13 + 4 * (D - 1))
    return closed, char


ALG_CLOSED_3D, ALG_FIXED_3D = alg_counts(3)
FP64_CLOSED_3D = ALG_CLOSED_3D - 6 * 12 - 4 * 3   # the closed form's flops on the FP64 pipe
ALG_PER_RECON_KEEP = 9
ALG_PER_RECON = 38
ALG_CUTOFF = 21
# A straightforward per-interface evaluation (projection of six points as
# 5x5 matrix products, ten reconstructions with their indicators and
# weights, back-projection): about 1450 flops + 45 divisions (reported for
# comparison; the kernels evaluate fewer).
STRAIGHTFORWARD_FLOPS_PER_IFACE_3D = 1495
STATE_BYTES_PER_CELL = 5 * 8


def _dist(backend: str = "nccl"):
    """One process per GPU under torchrun (RANK / WORLD_SIZE / MASTER_* from the
    environment); (None, 0, 1) without it."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    dist.init_process_group(backend=backend)
    return dist, rank, ws


def max_over_ranks(dist, ms: float, device) -> float:
    """The slowest rank's time (every rank gets it); ms itself without ranks."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, cells: int, steps: int, ms: float) -> float:
    """Gcell-updates/s of the whole job: every replica advances `cells` cells by
    `steps` steps in the max-over-ranks time `ms` (weak scaling)."""
    return world * cells * steps / (ms * 1e-3) / 1e9


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


FLUX_KERNEL_SOURCES = ("teno_cert.cuh", "teno_device.cuh", "teno_fixsum.cuh", "teno_flux.cuh", "teno_kernels.cu")


def _source_hash() -> str:
    """Hash of the sources the interface-flux kernel is built from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2003_09145_gb300", "csrc")
    for fn in FLUX_KERNEL_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fn.encode() + fh.read())
    return h.hexdigest()[:16]


def _traffic_per_launch():
    """DRAM bytes per flux-kernel launch at the benchmark size, from the committed
    ncu summary, if that was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "flux_kernel_traffic.txt")
    rec = {}
    try:
        with open(path) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip()
    except OSError:
        return None
    if rec.get("source_hash") != _source_hash():
        return None
    try:
        return float(rec["bytes_per_launch_256"])
    except (KeyError, ValueError):
        return None


def cpu_baseline(sample_n: int = 96, steps: int = 2) -> dict:
    """The oracle (plain FP64 C, OpenMP on all host cores) on a bounded sample of
    the same workload: `steps` RK3 steps of the same turbulence generator on a
    sample_n^3 box."""
    import oracle
    from paper_2003_09145_gb300 import inputs
    P = inputs.solenoidal_turbulence(n=sample_n)
    U = P.U0
    t0 = time.perf_counter()
    for _ in range(steps):
        dt = oracle.euler_dt(U, P.n, P.dx, 0.5)
        U = oracle.euler_rk3_step(U, P.n, P.dx, P.bc, dt)
    el = time.perf_counter() - t0
    cells = sample_n ** 3 * steps
    return {"value": cells / el / 1e9, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{steps} SSP-RK3 steps on a {sample_n}^3 box of the same turbulence generator "
                      f"({el:.1f} s wall)"}


def run_reference(args, rank: int) -> None:
    """The oracle as the reference arm: each step one RK3 step of a bounded
    sample (64^3 box) of the workload, on the host cores."""
    if rank != 0:
        return
    import oracle
    from paper_2003_09145_gb300 import inputs
    n = 64
    P = inputs.solenoidal_turbulence(n=n)
    U = P.U0
    for _ in range(args.warmup):
        U = oracle.euler_rk3_step(U, P.n, P.dx, P.bc, oracle.euler_dt(U, P.n, P.dx, 0.5))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = oracle.euler_rk3_step(U, P.n, P.dx, P.bc, oracle.euler_dt(U, P.n, P.dx, 0.5))
    el = time.perf_counter() - t0
    value = n ** 3 * args.steps / el / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": f"{n}^3 box per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{args.steps} RK3 steps on a {n}^3 box"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _keep_all_mask(scheme) -> int:
    """Magnitudes m at which chi_k >= C_T holds for every k by the bound
    chi_k >= 1/(3 (1 + max chi~)^6) (the kernel skips the cutoff test there)."""
    K = scheme.b_u - scheme.b_l
    thr = [scheme.H * (K / j - 1.0) for j in range(1, K)] + [scheme.H * 2.0 ** -53]
    mask = 0
    for c in range(1, K + 1):
        m = scheme.b_l + c
        if 3.0 * (1.0 + thr[c - 1]) ** 6 * float(f"1e-{m}") <= 1.0 - 1e-9:
            mask |= 1 << m
    return mask


def flux_classes(api, grid, U):
    """Per interface of U (from the flag path's selections): the number of its
    2 nvar reconstructions whose m lies outside the keep-all magnitudes (those
    evaluate the cutoff; an interface with none takes the closed form).
    Returns (algorithmic flops per interface, fraction of reconstructions that
    evaluate the cutoff, fraction of interfaces off the closed form)."""
    import torch
    _, fl = api.rhs(grid, U, want_flags=True)
    keep_all = _keep_all_mask(grid.scheme)
    nvar, ndim = grid.nvar, grid.ndim
    closed, char = alg_counts(ndim)
    alg_sum, nk_sum, off_sum, tot, off = 0.0, 0.0, 0.0, 0, 0
    for d in range(ndim):
        nifc_d = 1
        for k in range(ndim):
            nifc_d *= grid.n[k] + (1 if k == d else 0)
        blk = fl[off:off + nvar * 2 * nifc_d].view(nvar * 2, nifc_d)
        off += nvar * 2 * nifc_d
        nk = (((keep_all >> (blk >> 3).to(torch.int64)) & 1) == 0).sum(dim=0).double()
        per = torch.where(nk == 0, torch.full_like(nk, float(closed)),
                          char + 2 * nvar * ALG_PER_RECON_KEEP
                          + nk * (ALG_PER_RECON - ALG_PER_RECON_KEEP + ALG_CUTOFF))
        alg_sum += float(per.sum())
        nk_sum += float(nk.sum())
        off_sum += float((nk > 0).sum())
        tot += nifc_d
    del fl
    return alg_sum / tot, nk_sum / (2 * nvar * tot), off_sum / tot


def timed_steps(api, lib, solver, U, steps):
    """Event-timed `steps` RK3 steps of U; returns (ms per step, per-kind
    kernel ms and launch counts from the library's launch timer)."""
    import torch
    from paper_2003_09145_gb300 import _lib
    _lib.check(lib.teno_timer_begin(), "teno_timer_begin")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        solver.step(U)
    e1.record()
    torch.cuda.synchronize()
    kms = (ctypes.c_double * 4)()
    kcount = (ctypes.c_int64 * 4)()
    _lib.check(lib.teno_timer_end(kms, kcount), "teno_timer_end")
    return e0.elapsed_time(e1) / steps, dict(zip(_lib.KERNEL_KINDS, zip(list(kms), list(kcount))))


def bench_riemann2d(api, lib, device, steps: int, warm_steps: int, peak: float) -> dict:
    """The adaptive path at scale: the four-quadrant Riemann problem at 2048^2
    (split at (0.8, 0.8)), advanced `warm_steps` untimed steps so that its
    shocks, contacts and their interactions spread over the grid, then
    `steps` timed steps.  The roofline weights the closed-form and the
    characteristic-path counts by the classes of the timed start state."""
    import torch
    from paper_2003_09145_gb300 import inputs
    P = inputs.riemann_2d(n=2048)
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    solver = api.Solver(grid, device=device, cfl=0.5)
    U = torch.from_numpy(P.U0).to(device)
    solver.run(U, float("inf"), max_steps=warm_steps)
    torch.cuda.synchronize()
    assert solver.status() == 0
    t_start = float(solver.t.item())
    alg, cut, off = flux_classes(api, grid, U)
    ms, kinds = timed_steps(api, lib, solver, U, steps)
    flux_ms = kinds["flux"][0]
    nifc = (P.n[0] + 1) * P.n[1] + P.n[0] * (P.n[1] + 1)
    # one flux evaluation = both passes of one direction in one RK stage
    flux_s_per_step = flux_ms / steps * 1e-3
    achieved = alg * nifc * 3 / flux_s_per_step / 1e12
    return {"value": grid.ncell / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
            "workload": "2D four-quadrant Riemann problem (split (0.8, 0.8)), 2048^2, TENO5-LAD, SSP-RK3 "
                        f"CFL 0.5, timed from t = {t_start:.4f} (after {warm_steps} steps)",
            "interfaces_off_closed_form": off, "cutoff_evaluated_fraction": cut,
            "alg_flops_per_interface": alg,
            "kernel_ms_per_step": {k: v[0] / steps for k, v in kinds.items()},
            "flux_roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                              "frac": achieved / peak}}


def bench_schemes(api, lib, device, steps: int, workloads) -> dict:
    """The paper's cost comparison (Tab. 2) on this GPU: ms per RK3 step of
    the same state under TENO5-LAD and its comparison schemes (TENO5 with
    C_T = 1e-7, TENO5-A, WENO-Z), and the ratio to TENO5-LAD."""
    import torch
    out = {}
    for name, P, U0 in workloads:
        row = {}
        for sch in ("lad", "teno5", "teno5a", "wenoz"):
            grid = api.EulerGrid(P.n, P.dx, P.bc, api.Scheme(scheme=sch))
            solver = api.Solver(grid, device=device, cfl=0.5)
            U = U0.clone()
            for _ in range(2):
                solver.step(U)
            torch.cuda.synchronize()
            ms, _ = timed_steps(api, lib, solver, U, steps)
            assert solver.status() == 0
            row[sch] = {"ms_per_step": ms}
            del solver, U
            torch.cuda.empty_cache()
        for sch in row:
            row[sch]["vs_lad"] = row[sch]["ms_per_step"] / row["lad"]["ms_per_step"]
        out[name] = row
    out["paper_context"] = ("Tab. 2 (2D Euler, the paper's CPU workstation, seconds per step): TENO5-LAD about "
                            "1.05x TENO5, TENO5-A about 1.3x TENO5, WENO-Z about 0.9x TENO5")
    return out


# The paper's Tab. 2: average wall time of one time step (s) on its CPU
# workstation, per scheme (WENO-Z, TENO5, TENO5-A, TENO5-LAD).
PAPER_TAB2_S = {
    "rt128x512": {"wenoz": 0.14, "teno5": 0.15, "teno5a": 0.20, "lad": 0.16},
    "rt256x1024": {"wenoz": 0.59, "teno5": 0.67, "teno5a": 0.88, "lad": 0.70},
    "cfg3_1024": {"wenoz": 2.57, "teno5": 2.89, "teno5a": 3.71, "lad": 2.99},
    "cfg12_1024": {"wenoz": 2.56, "teno5": 2.85, "teno5a": 3.68, "lad": 2.99},
    "cfg12_2048": {"wenoz": 11.9, "teno5": 13.1, "teno5a": 17.8, "lad": 13.7},
}


def bench_tab2(api, device, max_steps_2048: int = 300) -> dict:
    """The paper's Tab. 2 workloads on this GPU: the Rayleigh-Taylor problem
    (Sec. 4.3.2) at 128x512 and 256x1024 to t = 1.95, the 2D Riemann
    configurations 3 (to t = 0.3) and 12 (to t = 0.25) at 1024^2, and
    configuration 12 at 2048^2 for its first `max_steps_2048` steps; each
    under the four schemes, ms per step averaged over the run (event-timed)
    beside the paper's seconds per step."""
    import torch
    from paper_2003_09145_gb300 import inputs
    cases = [("rt128x512", lambda: inputs.rayleigh_taylor(128, 512), None),
             ("rt256x1024", lambda: inputs.rayleigh_taylor(256, 1024), None),
             ("cfg3_1024", lambda: inputs.riemann_2d_config3(1024), None),
             ("cfg12_1024", lambda: inputs.riemann_2d_config12(1024), None),
             ("cfg12_2048", lambda: inputs.riemann_2d_config12(2048), max_steps_2048)]
    out = {}
    for name, make, cap in cases:
        P = make()
        row = {}
        for sch in ("lad", "teno5", "teno5a", "wenoz"):
            grid = api.EulerGrid(P.n, P.dx, P.bc, api.Scheme(gamma=P.gamma, scheme=sch), grav=P.extra.get("grav"),
                                 bc_state=P.extra.get("bc_state"))
            solver = api.Solver(grid, device=device, cfl=P.cfl)
            U = torch.from_numpy(P.U0).to(device)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            w0 = time.perf_counter()
            e0.record()
            k, limit, bad = 0, cap or 200000, None
            # in chunks, with a wall-clock budget per run (a run whose steps
            # shrink towards zero must not hold the GPU); a non-physical
            # state (the status word) ends the run
            while k < limit and float(solver.t.item()) < P.t_end and time.perf_counter() - w0 < 120.0:
                k += solver.run(U, P.t_end, max_steps=min(500, limit - k))
                if solver.status() != 0:
                    bad = {"by_step": k, "t": float(solver.t.item())}
                    break
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            print(f"tab2 {name} {sch}: {k} steps to t = {float(solver.t.item()):.4f}, {ms:.3f} ms/step",
                  file=sys.stderr, flush=True)
            row[sch] = {"steps": k, "t": float(solver.t.item()), "ms_per_step": ms,
                        "complete": bool(cap is not None or float(solver.t.item()) >= P.t_end),
                        "nonphysical": bad,
                        "paper_s_per_step": PAPER_TAB2_S[name][sch],
                        "speedup_vs_paper": PAPER_TAB2_S[name][sch] / (ms * 1e-3)}
            del solver, U
        out[name] = row
    return out


def fp64_probe(api, device) -> float:
    """Measured FP64 FMA throughput (flop/s) of this GPU."""
    import torch
    lib = api._lib.load()
    blocks, iters = SM_COUNT * 16, 4096
    out = torch.empty(blocks * 256, dtype=torch.float64, device=device)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        api._lib.check(lib.teno_probe_fp64(ctypes.c_void_p(out.data_ptr()), blocks, iters, st), "probe")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    api._lib.check(lib.teno_probe_fp64(ctypes.c_void_p(out.data_ptr()), blocks, iters, st), "probe")
    e1.record()
    torch.cuda.synchronize()
    return blocks * 256 * 8 * iters * 2 / (e0.elapsed_time(e1) * 1e-3)


def bench_batched(api, device, steps: int) -> dict:
    """The batched form on the 4096-tube workload (N log-uniform in [64, 4096],
    seed 20200320), every tube active: one persistent launch per RK stage,
    `steps` steps captured in one CUDA graph; beside it the same tubes advanced
    one by one through teno_rk3_step (one step each)."""
    import numpy as np
    import torch
    from paper_2003_09145_gb300 import autotune, inputs
    B = inputs.tube_batch(nprob=4096)
    solver = api.BatchSolver(B.n, B.dx, np.full(B.nprob, np.inf), device=device)
    U = torch.from_numpy(B.U0).to(device)
    tuning = autotune.tune_batched(solver, U, steps=2, use_cache=False)
    solver.capture(U, steps)
    solver.graph.replay()                       # warm-up replay
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    solver.graph.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # the same tubes one by one (single-problem path, one step each)
    singles = []
    for p in range(B.nprob):
        g = api.EulerGrid((int(B.n[p]),), (float(B.dx[p]),), (1,))
        singles.append((api.Solver(g, device=device),
                        torch.from_numpy(np.ascontiguousarray(B.U0[:, B.offsets[p]:B.offsets[p + 1]])).to(device)))
    for s_, u_ in singles[:8]:
        s_.step(u_)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for s_, u_ in singles:
        s_.step(u_)
    f1.record()
    torch.cuda.synchronize()
    ms_single = f0.elapsed_time(f1)
    return {"value": B.ncell / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
            "workload": "4096 independent shock tubes, N log-uniform in [64,4096] (sum N = %d), FP64" % B.ncell,
            "tuning": {"block": tuning[0], "ctas_per_sm": tuning[1]}, "graph_steps": steps,
            "one_by_one": {"value": B.ncell / (ms_single * 1e-3) / 1e9, "unit": UNIT,
                           "ms_per_step": ms_single}}


def bench_adjoint(api, device, grid, U0, steps: int) -> dict:
    """The adjoint form on the same 256^3 box: reverse of fixed-dt SSP-RK3 steps
    (teno_rk3_step_adjoint: two recomputed forward stages + three right-hand-side
    adjoints per step), reported like the forward path (cells x steps / time)."""
    import torch
    adj = api.AdjointStepper(grid, device=device)
    dt = 1e-3
    B = torch.ones_like(U0)
    adj.step(U0, dt, B, B)                      # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        adj.step(U0, dt, B, B)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    assert adj.status() == 0
    # the same reverse steps with the stages kept by the staged forward entry
    # points (teno_rk3_step_adjoint_staged: a rollout that replays its steps
    # keeps them; only the reverse step is timed)
    stages = api.rk3_step_stages(api.SlabEngine(grid, device=device), U0, dt)[:2]
    adj.step(U0, dt, B, B, stages=stages)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        adj.step(U0, dt, B, B, stages=stages)
    e1.record()
    torch.cuda.synchronize()
    ms_st = e0.elapsed_time(e1) / steps
    assert adj.status() == 0
    del stages
    return {"value": grid.ncell / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
            "workload": "reverse of one fixed-dt SSP-RK3 step on the 256^3 turbulence box, FP64",
            "stages_kept": {"value": grid.ncell / (ms_st * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms_st,
                            "how": "teno_rk3_step_adjoint_staged with the step's stages U1, U2 given"}}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_CELLS_1D, help="cells per axis (default 256)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched / adjoint / 2D / scheme forms")
    ap.add_argument("--form", choices=["riemann2d", "adjoint", "tab2"], default=None,
                    help="run only this form and print its record (profiling aid)")
    ap.add_argument("--warm-steps", type=int, default=400, help="untimed steps before the riemann2d form")
    args = ap.parse_args()

    dist, rank, world = _dist()
    if args.impl == "reference":
        run_reference(args, rank)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    import torch
    from paper_2003_09145_gb300 import api, inputs
    from paper_2003_09145_gb300 import _lib

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    lib = _lib.load()
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = SM_COUNT * FP64_FLOP_PER_CLK_PER_SM * sm_max * 1e6 / 1e12

    if args.form == "riemann2d":
        print(json.dumps(bench_riemann2d(api, lib, device, args.steps, args.warm_steps, peak)), flush=True)
        return
    if args.form == "tab2":
        print(json.dumps(bench_tab2(api, device)), flush=True)
        return
    if args.form == "adjoint":
        P = inputs.solenoidal_turbulence(n=args.n)
        grid = api.EulerGrid(P.n, P.dx, P.bc)
        print(json.dumps(bench_adjoint(api, device, grid, torch.from_numpy(P.U0).to(device), args.steps)),
              flush=True)
        return

    n = args.n
    P = inputs.solenoidal_turbulence(n=n)
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    solver = api.Solver(grid, device=device, cfl=0.5)
    U0 = torch.from_numpy(P.U0).to(device)
    U = U0.clone()
    t_end = float("inf")

    for _ in range(args.warmup):
        solver.step(U, t_end)
    torch.cuda.synchronize()
    assert solver.status() == 0, "non-physical state during warm-up"

    # algorithmic FP64 flops per interface on the timed start state: the flags
    # tell, per interface, how many of its ten reconstructions fall outside the
    # magnitudes m at which every stencil is provably kept
    alg_per_ifc, cut_frac, off_frac = flux_classes(api, grid, U)
    closed_frac = 1.0 - off_frac

    # ---- device-resident timed region --------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    _lib.check(lib.teno_timer_begin(), "teno_timer_begin")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        solver.step(U, t_end)
    e1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    kms = (ctypes.c_double * 4)()
    kcount = (ctypes.c_int64 * 4)()
    _lib.check(lib.teno_timer_end(kms, kcount), "teno_timer_end")
    clk = clocks.stop()
    assert solver.status() == 0, "non-physical state in the timed region"
    ms = max_over_ranks(dist, ms, device)
    cells = grid.ncell
    value = whole_job_rate(world, cells, args.steps, ms)

    # ---- roofline of the dominant kernel (interface fluxes) ----------------
    kinds = dict(zip(_lib.KERNEL_KINDS, zip(list(kms), list(kcount))))
    flux_ms, _ = kinds["flux"]
    # one flux evaluation per direction and RK stage: the closed-form pass and
    # the pass over the interfaces it leaves pending, timed together
    flux_evals = args.steps * 3 * 3
    nifc = (n + 1) * n * n
    flux_avg_s = flux_ms / flux_evals * 1e-3
    achieved = alg_per_ifc * nifc / flux_avg_s / 1e12
    probe = fp64_probe(api, device) / 1e12
    traffic = _traffic_per_launch()
    total_kernel_ms = sum(kms)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "flux_closed_kernel<3,d> + flux_pending_kernel<3,d> (interface fluxes, "
                          "one direction of one RK stage per evaluation)",
                "kernel_share": flux_ms / total_kernel_ms if total_kernel_ms else None,
                "peak_source": f"derived: {SM_COUNT} SMs x {FP64_FLOP_PER_CLK_PER_SM} FP64 flop/clk x "
                               f"{sm_max:.0f} MHz (max SM clock)",
                "fp64_probe_tflops": probe,
                "alg_flops_per_interface": alg_per_ifc,
                "fp64_flops_per_interface": alg_per_ifc - (ALG_CLOSED_3D - FP64_CLOSED_3D) * closed_frac,
                "fixed_point_sums": "closed form: the five M-weighted sums (60 U~) and the mass flux's "
                                    "P-weighted sum in 64-bit fixed point on the integer pipes (terms "
                                    "truncated 3 bits below the largest value's ulp, summed exactly, "
                                    "rounded once to binary64); the momentum and energy P-sums as "
                                    "binary64 chains",
                "cutoff_evaluated_fraction": cut_frac,
                "straightforward_count_tflops": STRAIGHTFORWARD_FLOPS_PER_IFACE_3D * nifc / flux_avg_s / 1e12}

    # ---- end to end through the public API with host buffers ---------------
    U_host = P.U0.copy()
    pin = torch.from_numpy(U_host).pin_memory()
    out_host = torch.empty_like(pin).pin_memory()
    solver.reset_time(0.0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # every step: H2D of its input, one RK3 step, D2H of its result; the copies
    # of neighbouring steps overlap the compute (api.HostPipeline)
    pipe = api.HostPipeline(solver, U0)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    pipe.run([pin] * args.steps, [out_host] * args.steps, t_end)
    f1.record()
    torch.cuda.synchronize()
    ems = f0.elapsed_time(f1)
    ems = max_over_ranks(dist, ems, device)
    nbytes = U0.numel() * 8
    e2e = {"value": whole_job_rate(world, cells, args.steps, ems), "unit": UNIT,
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
           "how": "api.HostPipeline: pinned H2D and D2H streams overlapping the steps"}

    forms = {}
    if not args.no_forms:
        forms["batched"] = bench_batched(api, device, max(args.steps, 4))
        forms["adjoint"] = bench_adjoint(api, device, grid, U0, 2)
        # the reverse step in forward steps of the timed region
        fwd_ms = ms / args.steps
        forms["adjoint"]["x_forward_step"] = forms["adjoint"]["ms_per_step"] / fwd_ms
        forms["adjoint"]["stages_kept"]["x_forward_step"] = forms["adjoint"]["stages_kept"]["ms_per_step"] / fwd_ms
        forms["riemann2d"] = bench_riemann2d(api, lib, device, max(args.steps, 5), args.warm_steps, peak)
        quad = inputs.riemann_2d(n=2048)
        qgrid = api.EulerGrid(quad.n, quad.dx, quad.bc)
        qsolver = api.Solver(qgrid, device=device, cfl=0.5)
        Uq = torch.from_numpy(quad.U0).to(device)
        qsolver.run(Uq, float("inf"), max_steps=args.warm_steps)
        del qsolver
        forms["schemes"] = bench_schemes(api, lib, device, 3,
                                         [("riemann2d_2048", quad, Uq), ("turbulence_256", P, U0)])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "cells": cells, "grid": [n, n, n],
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "l2": "inputs larger than L2 (state %.0f MB)" % (nbytes / 1e6)},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "forms": forms,
                "gpu_launches": int(sum(kcount)),
                "kernel_ms": {k: v[0] for k, v in kinds.items()},
                "clocks": clk, "impl": "ours"}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
