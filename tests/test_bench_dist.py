"""The multi-rank path of bench.py on CPU: world size 2 over gloo (127.0.0.1).

One process per GPU runs an independent replica (no collective on the data
path); the step time is the maximum over ranks and the reported value is the
whole-job rate.  The reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
import types
from contextlib import redirect_stdout

import pytest

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank's own step time; every rank learns the slowest
        mx = bench.ranks_max(values[rank], world, dist, "cpu")
        rate = bench.job_rate(1000.0, world, mx)
        out.put((rank, mx, rate))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    values = [0.25, 0.5]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, mx, rate in got:
        assert mx == 0.5
        assert rate == pytest.approx(2 * 1000.0 / 0.5)


def test_one_rank_needs_no_process_group():
    assert bench.ranks_max(0.125, 1, None, "cpu") == 0.125
    assert bench.job_rate(10.0, 1, 0.5) == 20.0


def test_reference_arm_is_rank_zero_only(monkeypatch):
    """A rank other than 0 exits 0 without work and prints nothing."""
    monkeypatch.setenv("RANK", "1")
    args = types.SimpleNamespace(steps=None, warmup=1, config="c2", gpus=2, k=0)
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args) == 0
    assert buf.getvalue() == ""
