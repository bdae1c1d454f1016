"""Multi-GPU form of the benchmark (replicas only: keys are independent, so
each rank runs its own batches with no data-path collective), checked on the
CPU as two gloo processes: disjoint key ranges give distinct keys (oracle),
the job time is the max over ranks, and the rate counts every rank's keys."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    import bench
    import oracle
    base = bench.replica_key_base(rank)
    pk, _, _ = oracle.keygen(761, 1, base)  # first key of this rank's range
    digest = torch.tensor(np.frombuffer(pk[:64].tobytes(), np.uint8).astype(np.int64))
    gathered = [torch.zeros_like(digest) for _ in range(world)]
    dist.all_gather(gathered, digest)
    t = bench.max_over_ranks(10.0 + rank, dist, "cpu")  # rank-dependent "step time"
    dist.barrier()
    out.put((rank, base, [g.tolist() for g in gathered], t))
    dist.destroy_process_group()


def test_replicas_two_gloo_ranks():
    import multiprocessing as mp
    import bench
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(out.get(timeout=240) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, b0, g0, t0), (r1, b1, g1, t1) = res
    assert b1 - b0 >= 1 << 40                      # disjoint key index ranges
    assert g0 == g1 and g0[0] != g0[1]            # the two ranks' first keys differ
    assert t0 == t1 == 11.0                       # the job time is the slowest rank's
    assert bench.whole_job_rate(2, 4096, 3, 0.006) == pytest.approx(2 * 4096 * 3 / 0.006)
