"""Host logic of the N > 1 benchmark path on CPU with gloo, world size 2: the
max-over-ranks timing, the whole-job aggregate of replicas, and the reference arm
printing on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_rank = 10.0 + 5.0 * rank               # rank 1 is slower
    value, ms = bench.aggregate_throughput(2.0e12, ms_rank, world)
    bench.barrier(world)
    # reference arm: rank 0 prints one line, the others exit without work
    sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0", "--size", "64"]
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.main()
    q.put((rank, value, ms, rc, buf.getvalue().strip()))
    dist.destroy_process_group()


def test_two_rank_timing_and_reference_arm():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, value, ms, rc, text = q.get(timeout=240)
        out[rank] = (value, ms, rc, text)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks agree on the slowest rank's time and on the aggregate
    assert out[0][1] == out[1][1] == 15.0
    assert abs(out[0][0] - 2 * 2.0e12 / 15.0e-3 / 1e12) < 1e-9
    assert out[0][2] == 0 and out[1][2] == 0
    assert '"impl": "reference"' in out[0][3]
    assert out[1][3] == ""
