"""Replica bookkeeping of bench.py with two gloo ranks on the CPU: the barrier,
the max over ranks of the timed region, the whole-job value as the sum of the
ranks' work over that max, and the reference arm running on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    got_ws, got_rank, _ = bench.dist_env()
    bench.barrier(ws)
    t = bench.max_over_ranks(ws, 1.0 + rank, "cpu")      # rank r's timed region: 1 + r seconds
    units_per_rank = 10.0
    value = ws * units_per_rank / t                       # whole-job value, as bench.py computes it
    dist.destroy_process_group()
    q.put((rank, got_ws, got_rank, t, value))


@pytest.mark.parametrize("ws", [2])
def test_two_rank_replica_timing(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got_ws, got_rank, t, value in out:
        assert got_ws == ws and got_rank == rank
        assert t == float(ws)                  # max over ranks
        assert abs(value - ws * 10.0 / ws) < 1e-12


def _ref_worker(rank, ws, port, q):
    import contextlib
    import io
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench

    class A:
        n = 12
        steps = 1
        warmup = 0
        method = "nat"
        k = 6

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(A())
    q.put((rank, buf.getvalue()))


def test_reference_arm_rank0_only():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_ref_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert '"impl": "reference"' in out[0]
    assert out[1] == ""
