"""Host-side multi-rank logic of the benchmark on CPU (gloo, world size 2): the
largest-first LPT split of a batch over ranks and the max-over-ranks reduction of the
step time.  Independent problems need no data-path collective, so these two are the
whole multi-GPU path."""
import multiprocessing as mp
import os
import socket

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1401_7962_gb300 import workloads as wl
    sizes = wl.diag_dominant_batch(1000, seed=5)[0]
    parts = bench.shard_lpt(sizes, world)
    t = bench.max_over_ranks(float(10 * (rank + 1)), world)
    bench.barrier(world)
    q.put((rank, t, parts[rank].tolist(), [len(p) for p in parts]))
    dist.destroy_process_group()


def test_two_rank_shard_and_max():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert all(o[1] == 20.0 for o in out)          # max over ranks seen by every rank
    import sys
    sys.path.insert(0, ROOT)
    from paper_1401_7962_gb300 import workloads as wl
    sizes = wl.diag_dominant_batch(1000, seed=5)[0]
    mine = [set(o[2]) for o in out]
    assert not (mine[0] & mine[1]) and (mine[0] | mine[1]) == set(range(len(sizes)))
    load = [float((sizes[list(m)].astype(np.float64) ** 3).sum()) for m in mine]
    assert abs(load[0] - load[1]) <= float(sizes.max()) ** 3   # LPT bound: one largest item
