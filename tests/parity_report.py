"""Parity report: the measured errors of the CUDA path against the oracle on
the five workload configurations (test infrastructure; run on a GPU machine
with ``python tests/parity_report.py``, prints a Markdown table).

The ``-m gpu`` tests assert the bounds (1e-12 relative max-norm for one
right-hand side, 1e-10 relative L1 after fixed step counts); this script
prints the values those tests bound, at the same sizes or larger.
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from oracle import grad  # noqa: E402
from paper_2003_09145_gb300 import api, inputs  # noqa: E402
from parity import compare_rhs, flux_scale, rel_l1_err, rel_max_err  # noqa: E402

ROWS = []


def row(config, quantity, value, bound, note=""):
    ROWS.append((config, quantity, value, bound, note))
    print(f"| {config} | {quantity} | {value} | {bound} | {note} |", flush=True)


def _oracle_extra(kw):
    out = {}
    if kw.get("grav") is not None:
        out["grav"] = tuple(kw["grav"]) + (0.0,) * (3 - len(kw["grav"]))
    if kw.get("bc_state") is not None:
        st = np.zeros((3, 2, 5))
        for k, faces in enumerate(kw["bc_state"]):
            if faces is not None:
                for side in range(2):
                    st[k, side, :len(faces[side])] = faces[side]
        out["bc_state"] = st
    return out


def rhs_pair(P, scheme=None, kw=None):
    grid = api.EulerGrid(P.n, P.dx, P.bc, scheme or api.Scheme(gamma=P.gamma), **(kw or {}))
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    a, fl = api.rhs(grid, U, want_flags=True)
    b = api.rhs(grid, U, want_flags=False)
    torch.cuda.synchronize()
    return a.cpu().numpy(), fl.cpu().numpy(), b.cpu().numpy()


def rhs_rows(name, P, scheme="lad", extra=None):
    kw = dict(extra or {})
    a, fl, b = rhs_pair(P, api.Scheme(gamma=P.gamma, scheme=scheme), kw)
    params = oracle.Params(gamma=P.gamma, scheme=scheme, **_oracle_extra(kw))
    err_a, rep = compare_rhs(P.U0, P.n, P.dx, P.bc, a, fl, oracle, params, max_examined=20000)
    err_b, _ = compare_rhs(P.U0, P.n, P.dx, P.bc, b, fl, oracle, params)
    fs = flux_scale(P.U0, P.n, P.dx, P.gamma)
    row(name, "one RHS, flag path: rel. max-norm", f"{err_a:.2e}", "1e-12")
    row(name, "one RHS, benchmark path (two-pass): rel. max-norm", f"{err_b:.2e}", "1e-12")
    row(name, "two paths against each other", f"{rel_max_err(b, a, fs):.2e}", "1e-13")
    row(name, "selection flags differing / total", f"{rep.mismatched} / {rep.total}",
        "counted", f"allowed delta {rep.allowed_delta}, m {rep.allowed_m}, unexplained {len(rep.unexplained)}")


def steps_row(name, P, steps, extra=None):
    kw = dict(extra or {})
    grid = api.EulerGrid(P.n, P.dx, P.bc, api.Scheme(gamma=P.gamma), **kw)
    solver = api.Solver(grid, cfl=P.cfl)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    for _ in range(steps):
        solver.step(U, P.t_end)
    Ug = U.cpu().numpy()
    Uo, t, k = oracle.euler_run(np.array(P.U0), P.n, P.dx, P.bc, P.t_end, sigma=P.cfl, max_steps=steps,
                                params=oracle.Params(gamma=P.gamma, **_oracle_extra(kw)))
    row(name, f"{k} RK3 steps (t = {t:.4g}): rel. L1", f"{rel_l1_err(Ug, Uo):.2e}", "1e-10",
        f"t GPU - t oracle = {solver.t.item() - t:.1e}")


def main():
    t0 = time.time()
    print("| config | quantity | measured | bound | note |")
    print("|---|---|---|---|---|")
    rhs_rows("1 Sod, N=200", inputs.shock_tube(200))
    steps_row("1 Sod, N=200", inputs.shock_tube(200), 400)
    rhs_rows("2 Shu-Osher, N=4096", inputs.shu_osher(4096))
    steps_row("2 Shu-Osher, N=4096", inputs.shu_osher(4096), 100)
    rhs_rows("3 four-quadrant, 2048^2", inputs.riemann_2d(n=2048))
    steps_row("3 four-quadrant, 2048^2", inputs.riemann_2d(n=2048, t_end=10.0), 20)
    for sch in ("teno5", "teno5a", "wenoz"):
        rhs_rows(f"3 four-quadrant, 2048^2, {sch}", inputs.riemann_2d(n=2048), scheme=sch)
    R = inputs.rayleigh_taylor(128, 512)
    rt = {"grav": R.extra["grav"], "bc_state": R.extra["bc_state"]}
    rhs_rows("Rayleigh-Taylor 128x512 (Sec. 4.3.2)", R, extra=rt)
    steps_row("Rayleigh-Taylor 128x512 (Sec. 4.3.2)", R, 20, extra=rt)

    # 4: batched tubes against the oracle, and bit for bit against single problems
    B = inputs.tube_batch(nprob=4096, seed=20200320)
    solver = api.BatchSolver(B.n, B.dx, np.full(B.nprob, 1e9))
    U = torch.from_numpy(B.U0).cuda()
    for _ in range(20):
        solver.step(U)
    Ug = U.cpu().numpy()
    rng = np.random.default_rng(0)
    worst, same = 0.0, 0
    picks = rng.choice(B.nprob, 24, replace=False)
    for p in picks:
        n = int(B.n[p])
        U0 = np.ascontiguousarray(B.U0[:, B.offsets[p]:B.offsets[p + 1]])
        Uo, _, _ = oracle.euler_run(U0, (n,), (B.dx[p],), (1,), 1e9, max_steps=20, strict=False)
        worst = max(worst, rel_l1_err(Ug[:, B.offsets[p]:B.offsets[p + 1]], Uo))
        g = api.EulerGrid((n,), (float(B.dx[p]),), (1,))
        s = api.Solver(g)
        Us = torch.from_numpy(U0.copy()).cuda()
        for _ in range(20):
            s.step(Us, 1e9)
        same += int(torch.equal(Us, U[:, B.offsets[p]:B.offsets[p + 1]]))
    row("4 batched, 4096 tubes", "20 RK3 steps, 24 sampled tubes: worst rel. L1", f"{worst:.2e}", "1e-10")
    row("4 batched, 4096 tubes", "sampled tubes equal to teno_rk3_step bit for bit", f"{same} / {len(picks)}",
        "all")

    # 5: 3D turbulence
    rhs_rows("5 turbulence, 256^3", inputs.solenoidal_turbulence(n=256))
    steps_row("5 turbulence, 256^3", inputs.solenoidal_turbulence(n=256, t_end=10.0), 2)
    P = inputs.solenoidal_turbulence(n=16)
    dt = oracle.euler_dt(P.U0, P.n, P.dx, 0.5)
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    U0 = torch.from_numpy(P.U0).cuda().requires_grad_(True)
    out = api.rollout(U0, grid, 40, dt, checkpoint_every=6)
    target = torch.from_numpy(inputs.perturbed_target(P.U0[0], seed=2)).cuda()
    loss = 0.5 * ((out[0] - target) ** 2).sum()
    loss.backward()
    Ut = torch.from_numpy(P.U0).requires_grad_(True)
    o = grad.rk3_rollout(Ut, P.n, P.dx, P.bc, dt, 40)
    lo = 0.5 * ((o[0] - torch.from_numpy(inputs.perturbed_target(P.U0[0], seed=2))) ** 2).sum()
    (g_or,) = torch.autograd.grad(lo, Ut)
    g_gpu = U0.grad.cpu().numpy()
    rel = np.linalg.norm(g_gpu - g_or.numpy()) / np.linalg.norm(g_or.numpy())
    row("5 adjoint, 16^3", "loss gradient after 40 steps (checkpoint 6): rel. L2", f"{rel:.2e}", "1e-10",
        f"loss rel. diff {abs(float(loss.detach()) - float(lo.detach())) / abs(float(lo.detach())):.1e}")
    print(f"\n({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    if not torch.cuda.is_available():
        sys.exit("parity_report needs a CUDA device")
    main()
