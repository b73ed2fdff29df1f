"""The multi-GPU form is replicas only: every rank holds the whole window and
draws its own walks, and the benchmark's whole-job figures are the summed
units over the slowest rank's time.  Checked with two gloo ranks on the CPU."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    hops = 1000 * (rank + 1)
    edges = 10 * (rank + 1)
    walk_s, ingest_s, total_ms = 1.0 + rank, 0.5 * (2 - rank), 100.0 + rank
    dist.barrier()
    r = bench.aggregate_ranks(hops, edges, walk_s, ingest_s, total_ms, world, device="cpu")
    out[rank] = (r, bench.rank_seed(rank))
    dist.destroy_process_group()


def test_two_replicas_aggregate_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, s0), (r1, s1) = out[0], out[1]
    assert r0 == r1 == (3000, 30, 2.0, 1.0, 101.0)  # summed units, slowest rank's times
    assert s0 != s1  # each replica draws its own walks
