"""Multi-GPU host logic on CPU: world_size 2 with the gloo backend.  The path shards by reads
with no data-path collective; ranks only agree on timing (max over ranks) and the whole-job
rate counts every rank's batch (weak scaling)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    ref, rd, params = bench.make_inputs(1, 0.01, r)
    slowest = bench.max_over_ranks(10.0 + rank, dist)
    rate = bench.whole_job_rate(ws, 3, rd.n, slowest * 3)
    q.put((rank, ws, int(ref.sum()), rd.seq[:64].tobytes(), slowest, rate, rd.n))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_reads_and_agree_on_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ws0, ref0, s0, t0, v0, n0), (r1, ws1, ref1, s1, t1, v1, n1) = out
    assert ws0 == ws1 == 2
    assert ref0 == ref1                 # one reference, replicated
    assert s0 != s1                     # each rank seeds its own reads
    assert t0 == t1 == 11.0             # both report the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 3 * n0 / (33.0 / 1000.0))
