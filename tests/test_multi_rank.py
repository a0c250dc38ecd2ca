"""The N > 1 path of the benchmark on CPU ranks (gloo, world size 2): every
rank holds the same dataset and held-out queries and its own disjoint slice
of the query batch (replicas: no data-path collective), the step time is the
maximum over ranks, and the reference arm runs on rank 0 only."""

import os
import socket
import time

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        bench.WORKLOAD.update(n=3000, m=24, nq=8, nheld=4)
        X, Q, H = bench.make_inputs(rank, world)
        items = [None] * world
        dist.all_gather_object(items, (X.tobytes(), Q.tobytes(), H.tobytes(), Q.shape))
        t = bench.reduce_max(1.5 * (rank + 1), world, "cpu")

        class Args:
            steps, warmup, cpu_c_alpha, B0, B, grow = 1, 0, 1e-2, 8, 8, 1
        ref = bench.run_reference(Args(), rank, world)
        if rank == 0:
            torch.save({"items": items, "t": t, "ref": ref is not None}, path)
        else:
            assert ref is None
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_shard_queries_and_take_the_slowest_time(tmp_path):
    world = 2
    path = str(tmp_path / "rank0.pt")
    port = _free_port()
    ctx = mp.start_processes(_rank_main, args=(world, port, path), nprocs=world, join=False, start_method="spawn")
    deadline = time.monotonic() + 240
    while not ctx.join(timeout=5):
        if time.monotonic() > deadline:
            for p in ctx.processes:
                p.terminate()
            raise AssertionError("ranks did not finish")
    res = torch.load(path)
    items, t, ref_on_rank0 = res["items"], res["t"], res["ref"]
    (x0, q0, h0, s0), (x1, q1, h1, s1) = items
    assert x0 == x1 and h0 == h1                 # the same dataset and held-out queries
    assert s0 == s1 == (8, 24) and q0 != q1      # disjoint query slices of equal size
    qa = np.frombuffer(q0, dtype=np.float32).reshape(8, 24)
    qb = np.frombuffer(q1, dtype=np.float32).reshape(8, 24)
    assert not any(np.array_equal(a, b) for a in qa for b in qb)
    assert t == 3.0                              # the slowest rank's time
    assert ref_on_rank0
