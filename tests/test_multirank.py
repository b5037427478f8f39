"""The N > 1 path of bench.py on CPU: world-size-2 gloo process groups.

Each rank solves its own problem (no collective on the data path); the only
collectives reduce the timed region to whole-job figures: the slowest rank's
time and the sum of the units all ranks processed.  The reference arm runs on
rank 0 alone."""
from __future__ import annotations

import contextlib
import io
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = bench.dist_info()
        # rank r "timed" 100 + 50 r ms over 259 + r matvecs
        ms, units = bench.reduce_over_ranks(100.0 + 50.0 * rank, 259 + rank, "cpu")
        q.put((rank, r, w, loc, ms, units))
    finally:
        dist.destroy_process_group()


def test_whole_job_figures_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, loc, ms, units in got:
        assert (r, w, loc) == (rank, 2, rank)
        assert ms == 150.0                 # the slowest rank's time
        assert units == 259.0 + 260.0      # every rank's matvecs
    # value = units / time: weak scaling over independent problems
    assert got[0][5] / (got[0][4] * 1e-3) == pytest.approx(519 / 0.150)


def test_single_process_keeps_its_own_figures():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.reduce_over_ranks(12.5, 30, "cpu") == (12.5, 30.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(A())
    assert out.getvalue() == ""            # rank 1 exits without work or output
