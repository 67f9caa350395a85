"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the path is
replicas only, so N > 1 runs one independent replica per rank; the timed
region's time is the max over ranks, `value` is the whole job's rate, and the
reference arm runs on rank 0 alone."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist, r, w = bench._dist(backend="gloo")
    assert (r, w) == (rank, world)
    ms = 10.0 + 5.0 * rank                     # rank 1 is the slower replica
    mx = bench.max_over_ranks(dist, ms, "cpu")
    rate = bench.whole_job_rate(w, 256 ** 3, 10, mx)
    # the reference arm: rank 0 alone does the work; other ranks return at once
    buf = io.StringIO()
    ran = None
    if rank != 0:
        with redirect_stdout(buf):
            ran = bench.run_reference(type("A", (), {"steps": 1, "warmup": 3, "gpus": world})(), rank)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, mx, rate, buf.getvalue(), ran))


def test_two_gloo_ranks_max_and_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, rate, printed, ran in res:
        assert mx == 15.0                       # the slowest rank's time, on every rank
        assert rate == pytest.approx(2 * 256 ** 3 * 10 / 15e-3 / 1e9)
    assert res[1][3] == "" and res[1][4] is None   # rank 1 printed nothing, did no work


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK") if k in os.environ}
    try:
        assert bench._dist() == (None, 0, 1)
    finally:
        os.environ.update(env)
    assert bench.max_over_ranks(None, 12.5, "cpu") == 12.5
    assert bench.whole_job_rate(1, 100, 2, 1000.0) == pytest.approx(2e-7)


def test_flop_accounting():
    """The roofline's per-interface counts, term by term as bench.py lists
    them: the closed form 187 (3D) / 153 (2D), the characteristic path 341 /
    290; of the closed form's 187, the FP64 pipe runs 103 (six of the ten
    six-point sums in fixed point: 72 FLOPs; the other four skip their
    products with weights +-1: 12)."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.alg_counts(3) == (187, 341)
    assert bench.alg_counts(2) == (153, 290)
    assert bench.ALG_CLOSED_3D - bench.FP64_CLOSED_3D == 6 * 12 + 4 * 3
    assert bench.FP64_CLOSED_3D == 103
    # the six-point sums are 12 algorithmic FLOPs each (one multiply-add per
    # point), ten per interface: 120 of the closed form's 187
    assert 10 * 12 == 6 * 4 * 5
