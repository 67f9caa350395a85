"""Autotuner for the batched kernel's launch shape (threads per CTA, persistent
CTAs per SM): each candidate is timed with CUDA events on copies of the state,
the fastest is kept and remembered in a JSON cache keyed by GPU name and batch
size."""
from __future__ import annotations

import json
import os

import torch

CANDIDATES = [(64, 4), (64, 8), (64, 16), (128, 2), (128, 4), (128, 8), (256, 1), (256, 2), (256, 4)]


def cache_path() -> str:
    return os.environ.get("TENO_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "teno_gb300", "autotune.json"))


def _key(solver) -> str:
    return f"batch:nprob={solver.nprob}:ncell={solver.ncell}"


def _load(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick_best(timings: dict) -> tuple:
    """The candidate with the smallest time (ties: the earlier candidate)."""
    best = None
    for cand, ms in timings.items():
        if best is None or ms < timings[best]:
            best = cand
    return best


def time_candidate(solver, U: torch.Tensor, cand, steps: int) -> float:
    """ms per step of ``steps`` batched steps with launch shape ``cand`` on a copy
    of U (the solver's times are restored afterwards)."""
    t_save = solver.t.clone()
    V = U.clone()
    solver.set_tuning(cand)
    solver.step(V)                      # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        solver.step(V)
    e1.record()
    torch.cuda.synchronize()
    solver.t.copy_(t_save)
    return e0.elapsed_time(e1) / steps


def tune_batched(solver, U: torch.Tensor, steps: int = 3, candidates=CANDIDATES, use_cache: bool = True,
                 timer=time_candidate) -> tuple:
    """Choose and apply the fastest (block, ctas_per_sm) for this solver."""
    gpu = torch.cuda.get_device_name(solver.device)
    path = cache_path()
    data = _load(path) if use_cache else {}
    hit = data.get(gpu, {}).get(_key(solver))
    if hit is not None:
        cand = tuple(hit["best"])
        solver.set_tuning(cand)
        return cand
    timings = {tuple(c): timer(solver, U, tuple(c), steps) for c in candidates}
    cand = pick_best(timings)
    solver.set_tuning(cand)
    if use_cache:
        data.setdefault(gpu, {})[_key(solver)] = {
            "best": list(cand), "ms_per_step": {f"{b}x{k}": v for (b, k), v in timings.items()}}
        _store(path, data)
    return cand
